"""GPU parity of the 1D column path (C ABI) against the CPU FP64 oracle.

Tolerances: float64 path 1e-12 relative (norm-wise and element-wise against the
largest reference entry); mixed apply 2e-5 relative (float32 Sigma and sweep:
a few hundred float32 roundings along a ray); solves to 1e-10 relative error
against the oracle's LU or GMRES solution.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2602_21958_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_APPLY_TOL = 2e-5


@pytest.fixture(scope="module")
def rt():
    from paper_2602_21958_gb300 import build_lib, rt as rtm

    build_lib.build()
    return rtm


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda:0")


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b), np.abs(a - b).max() / np.abs(b).max()


def small_problems():
    t = np.logspace(-3, 3, 13)
    return {
        "crd": W.two_level_column(t, 4, 1, 9, "crd", 1e-3, 1.0),
        "r2_ragged": W.two_level_column(np.logspace(-2, 4, 7), 6, 2, 11, "r2", 1e-4, 1.5),
        "mono_ie": W.paper_mono(10, 12),
        "iso_coh": W.paper_iso(8, 7, "coherent"),
        "iso_crd_ie": W.paper_iso(6, 5, "crd"),
        "dense": W.two_level_column(np.logspace(-2, 2, 6), 4, 2, 5, "r2", 1e-2, 1.0).with_dense_kernel(),
        "minimal": W.two_level_column(np.array([0.1, 2.0]), 2, 1, 1, "crd", 0.5, 1.0),
        "qsc": W.two_level_column(np.logspace(-3, 3, 17), 4, 2, 9, "r2", 1e-3, 1.0, formal_solver=W.FS_QSC),
        "qsc_short": W.two_level_column(np.array([0.05, 0.4, 3.0]), 2, 1, 3, "crd", 0.1, 1.0,
                                        formal_solver=W.FS_QSC),
    }


def oracle_op(p, op, x):
    if op == 0:
        return O.apply_A(p, x)
    if op == 1:
        return O.lambda_op(p, x)
    if op == 2:
        return O.sigma_op(p, x)
    return O.rhs(p)


@pytest.mark.parametrize("name", list(small_problems()))
@pytest.mark.parametrize("op", [0, 1, 2, 3])
def test_apply_fp64_parity(rt, name, op):
    p = small_problems()[name]
    h = rt.Handle(p, precision=rt.RT_P_FP64, max_restart=8)
    for seed, kind in ((0, "normal"), (1, "uniform")):
        x = W.random_vectors(p.n, 1, seed, kind)[0]
        y = torch.empty(p.n, dtype=torch.float64, device="cuda:0")
        h.rt_apply(op, dev(x), y)
        torch.cuda.synchronize()
        a, b = rel(y.cpu().numpy(), oracle_op(p, op, x))
        assert a < FP64_TOL and b < FP64_TOL, (name, op, a, b)


@pytest.mark.parametrize("name", ["crd", "r2_ragged", "dense", "iso_coh"])
def test_apply_mixed_error_bound(rt, name):
    p = small_problems()[name]
    h = rt.Handle(p, precision=rt.RT_P_MIXED, max_restart=8)
    x = W.random_vectors(p.n, 1, 3, "uniform")[0]
    y = torch.empty(p.n, dtype=torch.float64, device="cuda:0")
    h.rt_apply(0, dev(x), y)
    torch.cuda.synchronize()
    a, _ = rel(y.cpu().numpy(), O.apply_A(p, x))
    assert a < MIXED_APPLY_TOL, a


def test_ragged_batch_multi_rhs_apply(rt):
    probs = list(small_problems().values())
    n_rhs = 3
    h = rt.Handle(probs, n_rhs=n_rhs, precision=rt.RT_P_FP64, max_restart=8)
    E = sum(p.n for p in probs)
    assert h.length == n_rhs * E
    x = W.random_vectors(n_rhs * E, 1, 7)[0]
    y = torch.empty(n_rhs * E, dtype=torch.float64, device="cuda:0")
    h.rt_apply(0, dev(x), y)
    torch.cuda.synchronize()
    yc = y.cpu().numpy()
    for r in range(n_rhs):
        ref = O.apply_A_batch(probs, x[r * E:(r + 1) * E])
        a, b = rel(yc[r * E:(r + 1) * E], ref)
        assert a < FP64_TOL and b < FP64_TOL


def test_host_buffers_match_device_buffers(rt):
    p = small_problems()["r2_ragged"]
    h = rt.Handle(p, precision=rt.RT_P_FP64, max_restart=8)
    x = W.random_vectors(p.n, 1, 9)[0]
    y_host = np.empty(p.n)
    h.rt_apply(0, np.ascontiguousarray(x), y_host)
    y_dev = torch.empty(p.n, dtype=torch.float64, device="cuda:0")
    h.rt_apply(0, dev(x), y_dev)
    torch.cuda.synchronize()
    assert np.array_equal(y_host, y_dev.cpu().numpy())


# n_rhs = 1: one instance, solved by the grid-wide kernels; n_rhs = 2: two
# instances, one CTA each (the batched solve kernels)
@pytest.mark.parametrize("n_rhs", [1, 2])
@pytest.mark.parametrize("name", ["crd", "r2_ragged", "mono_ie", "iso_coh", "dense", "minimal", "qsc"])
def test_solve_fp64_matches_lu(rt, name, n_rhs):
    p = small_problems()[name]
    h = rt.Handle(p, n_rhs=n_rhs, precision=rt.RT_P_FP64, max_restart=64)
    b = O.rhs(p) if p.t_src is not None else np.ones(p.n)
    x = torch.zeros(n_rhs * p.n, dtype=torch.float64, device="cuda:0")
    info = h.rt_solve(dev(np.tile(b, n_rhs)), x, tol=1e-14, restart=64, max_outer=20)
    torch.cuda.synchronize()
    xref = np.linalg.solve(O.assemble_A(p), b)
    for r in range(n_rhs):
        a, _ = rel(x.cpu().numpy()[r * p.n:(r + 1) * p.n], xref)
        assert a < FP64_TOL * 10, (a, info)


@pytest.mark.parametrize("n_rhs", [1, 2])
@pytest.mark.parametrize("name", ["crd", "r2_ragged", "iso_coh", "dense", "qsc"])
def test_solve_mixed_refinement_matches_lu(rt, name, n_rhs):
    p = small_problems()[name]
    h = rt.Handle(p, n_rhs=n_rhs, precision=rt.RT_P_MIXED, max_restart=64)
    b = O.rhs(p)
    x = torch.zeros(n_rhs * p.n, dtype=torch.float64, device="cuda:0")
    info = h.rt_solve(dev(np.tile(b, n_rhs)), x, tol=1e-12, tol_inner=1e-4, restart=64, max_outer=30)
    torch.cuda.synchronize()
    assert info["status"] == 0, info
    xref = O.solve_dense(p)
    for r in range(n_rhs):
        a, _ = rel(x.cpu().numpy()[r * p.n:(r + 1) * p.n], xref)
        assert a < 1e-10, (a, info)


def test_batch_solve_internal_rhs_and_instances(rt):
    # columns with different formal solvers (SC-L, quadratic SC) in one batch
    probs = [small_problems()[k] for k in ("crd", "r2_ragged", "minimal", "qsc", "qsc_short")]
    n_rhs = 2
    E = sum(p.n for p in probs)
    h = rt.Handle(probs, n_rhs=n_rhs, precision=rt.RT_P_MIXED, max_restart=48)
    x = torch.zeros(n_rhs * E, dtype=torch.float64, device="cuda:0")
    info = h.rt_solve(None, x, tol=1e-12, tol_inner=1e-3, max_outer=40, per_instance=True)
    torch.cuda.synchronize()
    assert info["status"] == 0 and len(info["inst_relres"]) == n_rhs * len(probs)
    xc = x.cpu().numpy()
    ref = np.concatenate([O.solve_dense(p) for p in probs])
    for r in range(n_rhs):
        a, _ = rel(xc[r * E:(r + 1) * E], ref)
        assert a < 1e-10


def test_c1_full_size_solves(rt):
    """C1 (N = 10752): float64 GMRES and mixed refinement against the reduced
    CRD system solution (an independent oracle route)."""
    p = W.config_c1()
    xref = O.solve_crd_reduced(p)
    b = dev(O.rhs(p))
    for prec, extra in ((rt.RT_P_FP64, {}), (rt.RT_P_MIXED, {"tol_inner": 1e-4})):
        h = rt.Handle(p, precision=prec, max_restart=128)
        x = torch.zeros(p.n, dtype=torch.float64, device="cuda:0")
        # kappa(A) ~ 5e2 for C1: a residual of 1e-13 keeps the error below 1e-10
        info = h.rt_solve(b, x, tol=1e-13, restart=128, max_outer=30, **extra)
        torch.cuda.synchronize()
        a, _ = rel(x.cpu().numpy(), xref)
        assert info["status"] == 0 and a < 1e-10, (prec, a, info)


def test_c2_single_column_solves_meet_the_oracle_residual(rt):
    """C2 (131072 dofs, one column): the grid-wide routes (float64 GMRES, the
    nested mixed solve, BiCGStab) reach the tolerance on the oracle's own
    residual b - A x."""
    p = W.config_c2()
    b = O.rhs(p)
    bd = dev(b)
    cases = ((rt.RT_P_FP64, dict(restart=256)), (rt.RT_P_MIXED, dict(restart=64, tol_inner=0.1)),
             (rt.RT_P_FP64, dict(method=rt.RT_KRYLOV_BICGSTAB)))
    for prec, kw in cases:
        h = rt.Handle(p, precision=prec, max_restart=256 if prec == rt.RT_P_FP64 else 64)
        x = torch.zeros(p.n, dtype=torch.float64, device="cuda:0")
        info = h.rt_solve(bd, x, tol=1e-11, max_outer=80, **kw)
        torch.cuda.synchronize()
        assert info["status"] == 0, (prec, kw, info)
        r = np.linalg.norm(b - O.apply_A(p, x.cpu().numpy())) / np.linalg.norm(b)
        assert r < 2e-11, (prec, kw, r)


def test_c2_full_size_apply(rt):
    p = W.config_c2()
    x = W.random_vectors(p.n, 1, 11)[0]
    h = rt.Handle(p, precision=rt.RT_P_MIXED, max_restart=8)
    for fp64, tol in ((True, FP64_TOL), (False, MIXED_APPLY_TOL)):
        y = torch.empty(p.n, dtype=torch.float64, device="cuda:0")
        h.rt_apply(0, dev(x), y, fp64=fp64)
        torch.cuda.synchronize()
        a, _ = rel(y.cpu().numpy(), O.apply_A(p, x))
        assert a < tol, (fp64, a)


def test_c5_full_batch_apply_sampled_columns(rt):
    """Full C5 batch (256 columns x 4 rhs) in the launch configuration of the
    benchmark; the oracle recomputes a sample of (column, rhs) blocks."""
    cols = W.config_c5()
    n_rhs = 4
    E = sum(c.n for c in cols)
    h = rt.Handle(cols, n_rhs=n_rhs, precision=rt.RT_P_MIXED, max_restart=8)
    g = torch.Generator(device="cuda:0").manual_seed(5)
    x = torch.randn(n_rhs * E, dtype=torch.float64, device="cuda:0", generator=g)
    y64 = torch.empty_like(x)
    y32 = torch.empty_like(x)
    h.rt_apply(0, x, y64, fp64=True)
    h.rt_apply(0, x, y32, fp64=False)
    torch.cuda.synchronize()
    off = O.batch_offsets(cols)
    rng = np.random.default_rng(0)
    for ci in list(rng.choice(len(cols), 6, replace=False)) + [int(np.argmax([c.n for c in cols]))]:
        for r in (0, 3):
            sl = slice(r * E + off[ci], r * E + off[ci + 1])
            xc = x[sl].cpu().numpy()
            ref = O.apply_A(cols[ci], xc)
            a64, b64 = rel(y64[sl].cpu().numpy(), ref)
            a32, _ = rel(y32[sl].cpu().numpy(), ref)
            assert a64 < FP64_TOL and b64 < FP64_TOL and a32 < MIXED_APPLY_TOL, (ci, r, a64, a32)


def test_invalid_arguments_are_rejected(rt):
    p = small_problems()["crd"]
    bad = dataclasses.replace(p, z=p.z[::-1].copy())
    with pytest.raises(rt.RTError) as e:
        rt.Handle(bad)
    assert e.value.code == rt.RT_ERR_ARG
    nan = dataclasses.replace(p, chi=np.where(np.arange(p.chi.size).reshape(p.chi.shape) == 3, np.nan, p.chi))
    with pytest.raises(rt.RTError) as e:
        rt.Handle(nan)
    assert e.value.code == rt.RT_ERR_NONFINITE
    h = rt.Handle(p, max_restart=8)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda:0")
    with pytest.raises(rt.RTError) as e:
        h.rt_solve(None, x, restart=9)
    assert e.value.code == rt.RT_ERR_ARG


@pytest.mark.parametrize("n_rhs", [1, 2])
def test_nonfinite_rhs_reports_status(rt, n_rhs):
    p = small_problems()["crd"]
    h = rt.Handle(p, n_rhs=n_rhs, precision=rt.RT_P_FP64, max_restart=8)
    b = np.tile(O.rhs(p), n_rhs)
    b[5] = np.nan
    x = torch.zeros(n_rhs * p.n, dtype=torch.float64, device="cuda:0")
    info = h.rt_solve(dev(b), x, tol=1e-10, max_outer=3)
    assert info["status"] == rt.RT_ERR_NONFINITE


@pytest.mark.parametrize("n_rhs", [1, 2])
def test_iteration_count_reported_and_noconv(rt, n_rhs):
    p = W.config_c1()
    h = rt.Handle(p, n_rhs=n_rhs, precision=rt.RT_P_FP64, max_restart=4)
    x = torch.zeros(n_rhs * p.n, dtype=torch.float64, device="cuda:0")
    info = h.rt_solve(dev(np.tile(O.rhs(p), n_rhs)), x, tol=1e-12, restart=4, max_outer=2)
    assert info["status"] == rt.RT_ERR_NOCONV and info["max_outer"] == 2 and info["max_inner"] == 8


def test_repeated_solve_replays_identically(rt):
    """The batched solve is captured once into a CUDA graph and replayed while
    its arguments repeat; a replay must reproduce the first solve bit for bit,
    and changing an option must re-capture."""
    probs = [small_problems()[k] for k in ("crd", "r2_ragged")]
    h = rt.Handle(probs, n_rhs=2, precision=rt.RT_P_MIXED, max_restart=32)
    b = torch.tensor(np.concatenate([O.rhs_batch(probs)] * 2), device="cuda:0")
    x = torch.zeros_like(b)
    outs = []
    for tol in (1e-12, 1e-12, 1e-13):
        x.zero_()
        info = h.rt_solve(b, x, tol=tol, tol_inner=0.1, max_outer=40)
        torch.cuda.synchronize()
        assert info["status"] == 0
        outs.append(x.cpu().numpy().copy())
    assert np.array_equal(outs[0], outs[1])
    assert np.linalg.norm(outs[2] - outs[0]) <= 1e-10 * np.linalg.norm(outs[0])


def test_autotune_picks_a_shape_and_caches_it(rt, tmp_path, monkeypatch):
    """rt_autotune times the apply launch shapes, keeps the fastest (results
    unchanged: parity with the oracle after tuning), and a second handle of the
    same problem reads the choice from the RT_TUNE_CACHE file."""
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("RT_TUNE_CACHE", str(cache))
    probs = [small_problems()[k] for k in ("crd", "r2_ragged", "minimal")]
    h = rt.Handle(probs, n_rhs=2, precision=rt.RT_P_MIXED, max_restart=8)
    t = h.rt_autotune(force=True)
    assert t["ray_block"] in (64, 128, 256) and t["ahead"] in (2, 4, 8) and t["sigma_points"] in (4, 8, 0)
    assert not t["from_cache"] and t["ms_best"] > 0 and t["ms_best"] <= t["ms_default"] + 1e-9
    E = sum(p.n for p in probs)
    x = W.random_vectors(2 * E, 1, 61)[0]
    y = torch.empty(2 * E, dtype=torch.float64, device="cuda:0")
    h.rt_apply(0, dev(x), y, fp64=True)
    torch.cuda.synchronize()
    for r in range(2):
        ref = O.apply_A_batch(probs, x[r * E:(r + 1) * E])
        a, _ = rel(y.cpu().numpy()[r * E:(r + 1) * E], ref)
        assert a < FP64_TOL
    h2 = rt.Handle(probs, n_rhs=2, precision=rt.RT_P_MIXED, max_restart=8)
    t2 = h2.rt_autotune()
    assert t2["from_cache"] and (t2["ray_block"], t2["ahead"], t2["sigma_points"]) == \
        (t["ray_block"], t["ahead"], t["sigma_points"])


def test_autotune_persistent_solve_keeps_results_and_caches(rt, tmp_path, monkeypatch):
    """rt_autotune with the solve flag times the mixed batched solve's CTA
    shape (1 x 512 or 2 x 256 threads per SM) and inner cycle length; the
    solve afterwards (inner_restart = 0: the tuned length) still reaches the
    LU solution, and a second handle reads the choice from RT_TUNE_CACHE."""
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("RT_TUNE_CACHE", str(cache))
    probs = [small_problems()[k] for k in ("crd", "r2_ragged", "qsc", "minimal")]
    h = rt.Handle(probs, n_rhs=2, precision=rt.RT_P_MIXED, max_restart=32)
    t = h.rt_autotune(force=True, solve=True)
    assert t["solve_per_sm"] in (1, 2) and t["solve_inner"] in (12, 20, 30) and t["solve_ms"] > 0
    E = sum(p.n for p in probs)
    x = torch.zeros(2 * E, dtype=torch.float64, device="cuda:0")
    info = h.rt_solve(None, x, tol=1e-12, tol_inner=1e-2, max_outer=40, inner_restart=0)
    torch.cuda.synchronize()
    assert info["status"] == 0, info
    ref = np.concatenate([O.solve_dense(p) for p in probs])
    for r in range(2):
        a, _ = rel(x.cpu().numpy()[r * E:(r + 1) * E], ref)
        assert a < 1e-10
    h2 = rt.Handle(probs, n_rhs=2, precision=rt.RT_P_MIXED, max_restart=32)
    t2 = h2.rt_autotune(solve=True)
    assert t2["from_cache"] and (t2["solve_per_sm"], t2["solve_inner"]) == (t["solve_per_sm"], t["solve_inner"])
