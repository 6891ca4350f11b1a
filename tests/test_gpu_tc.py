"""GPU parity of the tensor-core (tcgen05, bf16 in / fp32 accumulate) Sigma for
dense kernels, through the C ABI (mixed-precision handles).

Two bars: (1) against the same contraction with X and Psi*w rounded to bf16
exactly as the kernel rounds them and summed in float64 -- the only remaining
difference is fp32 accumulation, bound 2e-6 relative; (2) against the float64
oracle, bound 1.5e-2 relative (bf16 operand rounding, 2^-8 per factor).
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


def bf16_round(a):
    """Round-to-nearest-even of float32 values to bf16, returned as float64."""
    f = np.asarray(a, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def emulated_sigma(p, x):
    """Gamma * (bf16(X) . bf16(PsiW)^T) with PsiW = Psi diag(w_dir (x) w_nu)."""
    wr = np.kron(p.w_dir, p.w_nu)
    psiw = bf16_round((p.Psi * wr[None, :]).astype(np.float32))
    X = bf16_round(x.astype(np.float32)).reshape(p.n_pts, p.n_r)
    C = X @ psiw.T
    g = np.tile(p.gamma.astype(np.float32).astype(np.float64), (1, p.n_dir))
    return (g * C).reshape(-1)


CASES = {
    "nr64": lambda: W.two_level_column(np.logspace(-2, 2, 9), 4, 2, 8, "r2", 1e-2, 1.0),
    "nr208_partial_chunk": lambda: W.two_level_column(np.logspace(-2, 3, 23), 4, 2, 26, "r2", 1e-3, 1.0),
    "nr320_ragged": lambda: W.two_level_column(np.logspace(-3, 3, 37), 8, 2, 20, "r2", 1e-3, 1.0),
    "nr1280": lambda: W.two_level_column(np.logspace(-4, 4, 150), 8, 2, 80, "r2", 1e-4, 1.0),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("n_rhs", [1, 3])
def test_tc_sigma_matches_bf16_emulation(rt, name, n_rhs):
    p = CASES[name]().with_dense_kernel()
    h = rt.Handle(p, n_rhs=n_rhs, precision=rt.RT_P_MIXED, max_restart=8)
    x = W.random_vectors(n_rhs * p.n, 1, 21)[0]
    y = torch.empty(n_rhs * p.n, dtype=torch.float64, device="cuda:0")
    h.rt_apply(rt.RT_OP_SIGMA, torch.tensor(x, device="cuda:0"), y)
    torch.cuda.synchronize()
    yc = y.cpu().numpy()
    for r in range(n_rhs):
        xs = x[r * p.n:(r + 1) * p.n]
        ys = yc[r * p.n:(r + 1) * p.n]
        ref = emulated_sigma(p, xs)
        assert np.linalg.norm(ys - ref) / np.linalg.norm(ref) < 2e-6
        orc = O.sigma_op(p, xs)
        assert np.linalg.norm(ys - orc) / np.linalg.norm(orc) < 1.5e-2


def test_tc_apply_A_and_fp64_override(rt):
    p = CASES["nr320_ragged"]().with_dense_kernel()
    h = rt.Handle(p, n_rhs=1, precision=rt.RT_P_MIXED, max_restart=8)
    x = W.random_vectors(p.n, 1, 22, "uniform")[0]
    xd = torch.tensor(x, device="cuda:0")
    y = torch.empty_like(xd)
    ref = O.apply_A(p, x)
    h.rt_apply(rt.RT_OP_A, xd, y)
    torch.cuda.synchronize()
    assert np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-2
    h.rt_apply(rt.RT_OP_A, xd, y, fp64=True)   # float64 operator on the same handle
    torch.cuda.synchronize()
    assert np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-12


def test_dense_mixed_solve_refines_to_fp64_accuracy(rt):
    """Mixed-precision handle with a dense kernel: the float64 refinement loop
    reaches the float64 solution (the solve kernel's inner operator takes the
    float32 CUDA-core Sigma)."""
    p = CASES["nr64"]().with_dense_kernel()
    h = rt.Handle(p, precision=rt.RT_P_MIXED, max_restart=64)
    b = torch.tensor(O.rhs(p), device="cuda:0")
    x = torch.zeros_like(b)
    info = h.rt_solve(b, x, tol=1e-13, tol_inner=1e-4, max_outer=40)
    torch.cuda.synchronize()
    xref = O.solve_dense(p)
    assert info["status"] == 0
    assert np.linalg.norm(x.cpu().numpy() - xref) / np.linalg.norm(xref) < 1e-10


def test_tc_timer_counts_and_times_only_the_gemm(rt):
    """rt_tc_timer brackets each tensor-core launch with CUDA events: three
    Sigma applies give three timed launches whose summed time is positive and
    below the applies' own (which also pack x to bf16); the output is the same
    as without a session, and ending a session that was never started is an
    argument error."""
    p = CASES["nr1280"]().with_dense_kernel()
    h = rt.Handle(p, n_rhs=2, precision=rt.RT_P_MIXED, max_restart=4)
    x = torch.tensor(W.random_vectors(2 * p.n, 1, 23)[0], device="cuda:0")
    y0 = torch.empty_like(x)
    y1 = torch.empty_like(x)
    h.rt_apply(rt.RT_OP_SIGMA, x, y0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h.rt_tc_timer(True)
    e0.record()
    for _ in range(3):
        h.rt_apply(rt.RT_OP_SIGMA, x, y1)
    e1.record()
    torch.cuda.synchronize()
    ms, n = h.rt_tc_timer(False)
    assert n == 3
    assert 0.0 < ms < e0.elapsed_time(e1)
    assert torch.equal(y0, y1)
    with pytest.raises(rt.RTError) as e:
        h.rt_tc_timer(False)
    assert e.value.code == rt.RT_ERR_ARG


def test_dense_single_column_mixed_solve_runs_sigma_on_the_tensor_cores(rt):
    """One dense column of 192,000 dofs in mixed precision is solved by the
    grid-wide nested solver, whose float32 inner operator takes the tcgen05
    Sigma: the kernel timer counts at least one tensor-core launch per inner
    iteration, and the float64 refinement still reaches the oracle's solution
    (the float64 outer operator closes every cycle)."""
    p = CASES["nr1280"]().with_dense_kernel()
    h = rt.Handle(p, precision=rt.RT_P_MIXED, max_restart=32)
    b = torch.tensor(O.rhs(p), device="cuda:0")
    x = torch.zeros_like(b)
    h.rt_tc_timer(True)
    info = h.rt_solve(b, x, tol=1e-12, tol_inner=1e-2, max_outer=40)
    torch.cuda.synchronize()
    ms, launches = h.rt_tc_timer(False)
    assert info["status"] == 0, info
    assert launches >= info["total_inner"] > 0 and ms > 0.0
    xref = O.solve_gmres(p, tol=1e-14, restart=400, max_iter=800).x
    assert np.linalg.norm(x.cpu().numpy() - xref) / np.linalg.norm(xref) < 1e-10
