"""The N > 1 bench path on CPU (gloo, world size 2): process-group set-up from
the torchrun environment, the max-over-ranks timing reduction, the barrier,
and that every rank builds its own seeded C5 batch (independent replicas, no
data-path collective)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RT_BENCH_BACKEND": "gloo"})
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import torch.distributed as dist

    r, w = bench.dist_setup()
    assert (r, w) == (rank, world)
    t = bench.dist_max(10.0 + rank, w)          # each rank's time -> the slowest
    bench.dist_barrier(w)
    cols = bench.workload(r)
    sig = np.array([[c.nz, c.n_nu] for c in cols[:8]], dtype=float).ravel()
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.concatenate([[t], sig]))
    dist.destroy_process_group()


def test_two_rank_gloo_bench_path(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    assert r0[0] == r1[0] == 11.0                # max over ranks on every rank
    assert not np.array_equal(r0[1:], r1[1:])    # distinct batches per rank
    from paper_2602_21958_gb300 import workloads as W
    ref = W.config_c5()
    assert np.array_equal(r0[1:], np.array([[c.nz, c.n_nu] for c in ref[:8]], dtype=float).ravel())
