"""Failure detection without a GPU fault: host-side injection (RT_FAULT) and a
bounded device wait that gives up.

* stall: the pipeline waits of the tensor-core Sigma poll once, give up,
  drain their own copies and MMAs, free tensor memory; the call returns
  RT_ERR_TIMEOUT and the handle then gives the right result.
* launch / nan_input / alloc: the calls return RT_ERR_CUDA, RT_ERR_NONFINITE
  (solve status filled), RT_ERR_OOM without launching anything.
"""
import numpy as np
import pytest

import oracle as O
from paper_2602_21958_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    from paper_2602_21958_gb300 import build_lib, rt as rtm

    build_lib.build()
    return rtm


def _dense_tc():
    return W.two_level_column(np.logspace(-2, 2, 33), 4, 2, 16, "r2", 1e-2, 1.0).with_dense_kernel()


def test_stalled_tensor_core_wait_times_out_and_the_handle_recovers(rt, monkeypatch):
    p = _dense_tc()
    h = rt.Handle(p, n_rhs=2, precision=rt.RT_P_MIXED, max_restart=4)
    x = torch.tensor(W.random_vectors(h.length, 1, 5)[0], device="cuda:0")
    y = torch.empty_like(x)
    monkeypatch.setenv("RT_FAULT", "stall")
    for op in (rt.RT_OP_SIGMA, rt.RT_OP_A):
        with pytest.raises(rt.RTError) as e:
            h.rt_apply(op, x, y)
        assert e.value.code == rt.RT_ERR_TIMEOUT, str(e.value)
    monkeypatch.delenv("RT_FAULT")
    h.rt_apply(rt.RT_OP_SIGMA, x, y)
    torch.cuda.synchronize()
    xc, yc = x.cpu().numpy(), y.cpu().numpy()
    for r in range(2):
        ref = O.sigma_op(p, xc[r * p.n:(r + 1) * p.n])
        assert np.linalg.norm(yc[r * p.n:(r + 1) * p.n] - ref) <= 1.5e-2 * np.linalg.norm(ref)
    # the float64 operator never waits on the pipeline: unaffected by the stall
    monkeypatch.setenv("RT_FAULT", "stall")
    h.rt_apply(rt.RT_OP_SIGMA, x, y, fp64=True)
    torch.cuda.synchronize()
    ref = O.sigma_op(p, xc[:p.n])
    assert np.linalg.norm(y.cpu().numpy()[:p.n] - ref) <= 1e-12 * np.linalg.norm(ref)


def test_injected_launch_nan_and_alloc_failures(rt, monkeypatch):
    p = W.two_level_column(np.logspace(-2, 2, 9), 4, 2, 8, "r2", 1e-2, 1.0)
    h = rt.Handle(p, n_rhs=2, precision=rt.RT_P_MIXED, max_restart=16)
    x = torch.zeros(h.length, dtype=torch.float64, device="cuda:0")
    y = torch.empty_like(x)
    monkeypatch.setenv("RT_FAULT", "launch")
    with pytest.raises(rt.RTError) as e:
        h.rt_apply(rt.RT_OP_A, x, y)
    assert e.value.code == rt.RT_ERR_CUDA
    with pytest.raises(rt.RTError) as e:
        h.rt_solve(None, x)
    assert e.value.code == rt.RT_ERR_CUDA
    monkeypatch.setenv("RT_FAULT", "nan_input")
    info = h.rt_solve(None, x)
    assert info["status"] == rt.RT_ERR_NONFINITE
    monkeypatch.setenv("RT_FAULT", "alloc")
    with pytest.raises(rt.RTError) as e:
        rt.Handle(p)
    assert e.value.code == rt.RT_ERR_OOM
    monkeypatch.delenv("RT_FAULT")
    info = h.rt_solve(None, x, tol=1e-12, tol_inner=1e-2, max_outer=40)
    assert info["status"] == rt.RT_OK
    ref = O.solve_dense(p)
    assert np.linalg.norm(x.cpu().numpy()[:p.n] - ref) <= 1e-10 * np.linalg.norm(ref)
