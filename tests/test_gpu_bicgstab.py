"""GPU BiCGStab (float64, the paper's second Krylov solver, Sec. 5) through the
C ABI, against the oracle: dense LU for 1D columns (batched, several rhs, both
handle precisions) and the oracle's own BiCGStab / GMRES for a 3D box; plus the
workspace check, the iteration cap and agreement with the GPU GMRES."""
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


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def columns():
    return [W.two_level_column(np.logspace(-3, 3, 13), 4, 1, 9, "crd", 1e-3, 1.0),
            W.two_level_column(np.logspace(-2, 4, 7), 6, 2, 11, "r2", 1e-4, 1.5),
            W.paper_iso(8, 7, "coherent"),
            W.two_level_column(np.array([0.1, 2.0]), 2, 1, 1, "crd", 0.5, 1.0)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_bicgstab_matches_lu(rt, prec):
    probs = columns()
    n_rhs = 3
    E = sum(p.n for p in probs)
    rng = np.random.default_rng(5)
    B = rng.standard_normal((n_rhs, E))
    h = rt.Handle(probs, n_rhs=n_rhs, precision=rt.RT_P_FP64 if prec == "fp64" else rt.RT_P_MIXED,
                  max_restart=8)
    x = torch.zeros(n_rhs * E, dtype=torch.float64, device="cuda:0")
    b = torch.tensor(B.ravel(), device="cuda:0")
    info = h.rt_solve(b, x, tol=1e-13, max_outer=10, method=rt.RT_KRYLOV_BICGSTAB, per_instance=True)
    torch.cuda.synchronize()
    assert info["status"] == 0, info
    assert info["max_relres"] <= 1e-13
    xc = x.cpu().numpy().reshape(n_rhs, E)
    offs = np.concatenate([[0], np.cumsum([p.n for p in probs])])
    for r in range(n_rhs):
        for i, p in enumerate(probs):
            xref = np.linalg.solve(O.assemble_A(p), B[r, offs[i]:offs[i + 1]])
            assert rel(xc[r, offs[i]:offs[i + 1]], xref) < 1e-10


def test_bicgstab_iterations_follow_the_oracle(rt):
    # same algorithm in the same arithmetic: the iteration counts to a modest
    # tolerance agree within a few steps (BiCGStab amplifies the different
    # rounding order of the sums: 92 against 96 measured)
    p = W.config_c1()
    b = O.rhs(p)
    ref = O.bicgstab(lambda v: O.apply_A(p, v), b, tol=1e-10)
    h = rt.Handle(p, precision=rt.RT_P_FP64, max_restart=8)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda:0")
    info = h.rt_solve(torch.tensor(b, device="cuda:0"), x, tol=1e-10, max_outer=10,
                      method=rt.RT_KRYLOV_BICGSTAB)
    torch.cuda.synchronize()
    assert info["status"] == 0
    assert abs(info["max_inner"] - ref.iterations) <= max(3, ref.iterations // 10), \
        (info["max_inner"], ref.iterations)
    assert rel(x.cpu().numpy(), O.solve_dense(p)) < 1e-7


def test_bicgstab_agrees_with_gpu_gmres_on_c5_columns(rt):
    probs = [W.config_c5_column(ci) for ci in (3, 100, 200)]
    E = sum(p.n for p in probs)
    h = rt.Handle(probs, n_rhs=1, precision=rt.RT_P_MIXED, max_restart=32)
    xg = torch.zeros(E, dtype=torch.float64, device="cuda:0")
    xb = torch.zeros_like(xg)
    ig = h.rt_solve(None, xg, tol=1e-13, tol_inner=0.1, restart=32, max_outer=60, inner_restart=20)
    ib = h.rt_solve(None, xb, tol=1e-13, max_outer=20, method=rt.RT_KRYLOV_BICGSTAB)
    torch.cuda.synchronize()
    assert ig["status"] == 0 and ib["status"] == 0, (ig, ib)
    assert rel(xb.cpu().numpy(), xg.cpu().numpy()) < 1e-9


def test_bicgstab_box_matches_oracle(rt):
    rng = np.random.Generator(np.random.PCG64(3))
    nx, ny, nz, n_nu, eps = 6, 5, 6, 5, 1e-3
    kappa = W.lognormal_opacity((nz, ny, nx), 1.5, rng, kappa0=0.7).ravel()
    dirs, wd = W.level_symmetric(4)
    xg, wn, phi, R = W.line_data(n_nu, "r2")
    npts = nx * ny * nz
    p = W.Problem(dims=3, nx=nx, ny=ny, nz=nz, z=np.array([1.0, 1.3, 0.8]), dirs=dirs, w_dir=wd, w_nu=wn,
                  chi=kappa[:, None] * phi[None, :], gamma=np.tile((1 - eps) / phi, (npts, 1)),
                  P=W.dipole_3d(dirs), R=R, t_src=np.full((npts, n_nu), eps),
                  I_top=np.zeros(n_nu), I_bot=np.ones(n_nu), formal_solver=W.FS_SCL)
    xref = O.solve_gmres(p, tol=1e-14, restart=300, max_iter=600).x
    for prec, m in ((rt.RT_P_FP64, 6), (rt.RT_P_MIXED, 12)):
        h = rt.Handle(p, precision=prec, max_restart=m)
        x = torch.zeros(p.n, dtype=torch.float64, device="cuda:0")
        info = h.rt_solve(None, x, tol=1e-13, max_outer=10, method=rt.RT_KRYLOV_BICGSTAB)
        torch.cuda.synchronize()
        assert info["status"] == 0, info
        assert rel(x.cpu().numpy(), xref) < 1e-10


def test_bicgstab_workspace_and_iteration_cap(rt):
    p = columns()[1]
    h = rt.Handle(p, precision=rt.RT_P_FP64, max_restart=2)  # 3 vectors: too few
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda:0")
    with pytest.raises(rt.RTError) as e:
        h.rt_solve(None, x, tol=1e-12, method=rt.RT_KRYLOV_BICGSTAB)
    assert e.value.code == rt.RT_ERR_ARG
    with pytest.raises(rt.RTError):
        h.rt_solve(None, x, tol=1e-12, method=7)
    h2 = rt.Handle(p, precision=rt.RT_P_FP64, max_restart=8)
    info = h2.rt_solve(None, x, tol=1e-14, max_outer=1, method=rt.RT_KRYLOV_BICGSTAB, max_iter=2)
    torch.cuda.synchronize()
    assert info["status"] == rt.RT_ERR_NOCONV and info["max_inner"] == 2
    # the reported residual is the true one, b - A x
    xr = x.cpu().numpy()
    b = O.rhs(p)
    true = np.linalg.norm(b - O.apply_A(p, xr)) / np.linalg.norm(b)
    assert abs(info["max_relres"] - true) <= 1e-9 * true
