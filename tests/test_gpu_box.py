"""GPU parity of the 3D box path (short-characteristics plane sweep, grid-wide
GMRES) against the CPU oracle.  Boxes are non-cubic with unequal spacings so
a transposed index or a swapped shift fails; float64 bar 1e-12, mixed apply
2e-5, solves 1e-10 against the oracle's own GMRES at 1e-14."""
import dataclasses
import math

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


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda:0")


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def small_box(nx=7, ny=5, nz=6, order=4, n_nu=6, kernel="crd", eps=1e-2, seed=1, spacing=(1.0, 1.3, 0.8)):
    rng = np.random.Generator(np.random.PCG64(seed))
    kappa = W.lognormal_opacity((nz, ny, nx), 1.5, rng, kappa0=0.7).ravel()
    dirs, wd = W.level_symmetric(order)
    x, wn, phi, R = W.line_data(n_nu, kernel)
    npts = nx * ny * nz
    return W.Problem(dims=3, nx=nx, ny=ny, nz=nz, z=np.array(spacing), dirs=dirs, w_dir=wd, w_nu=wn,
                     chi=kappa[:, None] * phi[None, :], gamma=np.tile((1 - eps) / phi, (npts, 1)),
                     P=W.dipole_3d(dirs), R=R, t_src=np.full((npts, n_nu), eps),
                     I_top=np.zeros(n_nu), I_bot=np.ones(n_nu), formal_solver=W.FS_SCL)


def oracle_op(p, op, x):
    return [O.apply_A, O.lambda_op, O.sigma_op][op](p, x) if op < 3 else O.rhs(p)


@pytest.mark.parametrize("op", [0, 1, 2, 3])
@pytest.mark.parametrize("variant", ["crd", "r2_ie", "dense"])
def test_box_apply_fp64(rt, op, variant):
    if variant == "crd":
        p = small_box()
    elif variant == "r2_ie":
        p = dataclasses.replace(small_box(n_nu=9, kernel="r2", nx=5, ny=8), formal_solver=W.FS_IE)
    else:
        p = small_box(nx=4, ny=3, nz=5, n_nu=4).with_dense_kernel()
    h = rt.Handle(p, precision=rt.RT_P_FP64, max_restart=8)
    x = W.random_vectors(p.n, 1, 30 + op)[0]
    y = torch.empty(p.n, dtype=torch.float64, device="cuda:0")
    h.rt_apply(op, dev(x), y)
    torch.cuda.synchronize()
    ref = oracle_op(p, op, x)
    assert rel(y.cpu().numpy(), ref) < 1e-12
    assert np.abs(y.cpu().numpy() - ref).max() < 1e-12 * np.abs(ref).max()


def test_box_apply_mixed_bound(rt):
    p = small_box(nx=9, ny=8, nz=7, order=6, n_nu=10, kernel="r2")
    h = rt.Handle(p, precision=rt.RT_P_MIXED, max_restart=8)
    x = W.random_vectors(p.n, 1, 40, "uniform")[0]
    y = torch.empty(p.n, dtype=torch.float64, device="cuda:0")
    h.rt_apply(0, dev(x), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), O.apply_A(p, x)) < 2e-5


def test_box_integer_offset_direction(rt):
    """A diagonal direction whose upwind point is exactly one cell back."""
    p = small_box(nx=6, ny=6, nz=5, spacing=(1.0, 1.0, 1.0))
    d = np.array([[1 / math.sqrt(2), 0.0, -1 / math.sqrt(2)], [0.0, -1 / math.sqrt(2), 1 / math.sqrt(2)]])
    p = dataclasses.replace(p, dirs=d, w_dir=np.array([0.5, 0.5]), P=np.ones((2, 2)))
    h = rt.Handle(p, precision=rt.RT_P_FP64, max_restart=8)
    x = W.random_vectors(p.n, 1, 41)[0]
    y = torch.empty(p.n, dtype=torch.float64, device="cuda:0")
    h.rt_apply(1, dev(x), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), O.lambda_op(p, x)) < 1e-13


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_box_solve(rt, prec):
    p = small_box(nx=6, ny=5, nz=6, order=4, n_nu=5, kernel="r2", eps=1e-3)
    xref = O.solve_gmres(p, tol=1e-14, restart=300, max_iter=600).x
    h = rt.Handle(p, precision=rt.RT_P_FP64 if prec == "fp64" else rt.RT_P_MIXED, max_restart=120)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda:0")
    info = h.rt_solve(None, x, tol=1e-13, tol_inner=1e-5, restart=120, max_outer=30)
    torch.cuda.synchronize()
    assert info["status"] == 0, info
    assert rel(x.cpu().numpy(), xref) < 1e-10


def test_c3_physics_reduced_grid(rt):
    """C3 physics (S_6, dipole x CRD, lognormal opacity, eps = 1e-3) on a
    10^3 box with 8 frequencies: mixed solve against the oracle."""
    p = W.box_3d(10, 6, 8, "crd", 1e-3, W.SEED_BASE + 3)
    xref = O.solve_gmres(p, tol=1e-13, restart=200, max_iter=400).x
    h = rt.Handle(p, precision=rt.RT_P_MIXED, max_restart=100)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda:0")
    info = h.rt_solve(None, x, tol=1e-12, tol_inner=1e-5, restart=100, max_outer=30)
    torch.cuda.synchronize()
    assert info["status"] == 0, info
    assert rel(x.cpu().numpy(), xref) < 1e-10


def nonseparable_box(seed=3, **kw):
    """small_box with chi(p, nu) = kappa(p) phi(nu) times an independent factor
    in [0.5, 1.5] per (point, frequency): the sweeps then read the full opacity
    instead of one kappa per cell."""
    p = small_box(seed=seed, **kw)
    rng = np.random.Generator(np.random.PCG64(seed + 100))
    return dataclasses.replace(p, chi=p.chi * rng.uniform(0.5, 1.5, p.chi.shape))


@pytest.mark.parametrize("coef64", ["precomputed", "on_the_fly"])
@pytest.mark.parametrize("separable", [True, False])
@pytest.mark.parametrize("op", [0, 1, 3])
def test_box_step_weight_modes_fp64(rt, monkeypatch, coef64, separable, op):
    """Every float64 step-weight mode of the plane sweep (precomputed per
    (direction, point, nu), or formed from the opacity) on separable and
    non-separable opacities, against the oracle."""
    if coef64 == "on_the_fly":
        monkeypatch.setenv("RT_BOX_COEF64", "0")
    kw = dict(nx=6, ny=7, nz=5, n_nu=7, kernel="r2")
    p = nonseparable_box(**kw) if not separable else small_box(seed=3, **kw)
    h = rt.Handle(p, precision=rt.RT_P_FP64, max_restart=4)
    x = W.random_vectors(p.n, 1, 50 + op)[0]
    y = torch.empty(p.n, dtype=torch.float64, device="cuda:0")
    h.rt_apply(op, dev(x), y)
    torch.cuda.synchronize()
    ref = oracle_op(p, op, x)
    assert rel(y.cpu().numpy(), ref) < 1e-12
    assert np.abs(y.cpu().numpy() - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("op", [0, 1])
def test_box_nonseparable_opacity_mixed(rt, op):
    """The float32 sweep with the full (blocked) opacity: apply within the
    mixed-apply bar."""
    p = nonseparable_box(nx=9, ny=8, nz=7, order=6, n_nu=10, kernel="r2")
    h = rt.Handle(p, precision=rt.RT_P_MIXED, max_restart=8)
    x = W.random_vectors(p.n, 1, 60 + op, "uniform")[0]
    y = torch.empty(p.n, dtype=torch.float64, device="cuda:0")
    h.rt_apply(op, dev(x), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), oracle_op(p, op, x)) < 2e-5


def test_box_nonseparable_opacity_mixed_solve(rt):
    p = nonseparable_box(nx=6, ny=5, nz=6, order=4, n_nu=5, kernel="r2", eps=1e-3)
    xref = O.solve_gmres(p, tol=1e-14, restart=300, max_iter=600).x
    h = rt.Handle(p, precision=rt.RT_P_MIXED, max_restart=120)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda:0")
    info = h.rt_solve(None, x, tol=1e-13, tol_inner=1e-5, restart=120, max_outer=30)
    torch.cuda.synchronize()
    assert info["status"] == 0, info
    assert rel(x.cpu().numpy(), xref) < 1e-10


@pytest.mark.parametrize("fb", ["1", "2", "4"])
@pytest.mark.parametrize("n_nu,kernel", [(8, "r2"), (12, "crd")])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_box_sigma_four_frequencies_per_lane(rt, monkeypatch, fb, n_nu, kernel, prec):
    """Frequency counts that are multiples of 4 take the Sigma kernel with four
    consecutive frequencies per lane and several points per warp; every sweep
    block width (RT_BOX_FB) and both precisions, all four operators."""
    monkeypatch.setenv("RT_BOX_FB", fb)
    p = small_box(nx=7, ny=6, nz=5, order=4, n_nu=n_nu, kernel=kernel, seed=9)
    h = rt.Handle(p, precision=rt.RT_P_FP64 if prec == "fp64" else rt.RT_P_MIXED, max_restart=4)
    for op in (0, 1, 2, 3):
        x = W.random_vectors(p.n, 1, 70 + op, "uniform")[0]
        y = torch.empty(p.n, dtype=torch.float64, device="cuda:0")
        h.rt_apply(op, dev(x), y)
        torch.cuda.synchronize()
        ref = oracle_op(p, op, x)
        bar = 1e-12 if prec == "fp64" else 2e-5
        assert rel(y.cpu().numpy(), ref) < bar, (op, fb)


def qsc_box(separable=True, **kw):
    p = small_box(**kw) if separable else nonseparable_box(**kw)
    return dataclasses.replace(p, formal_solver=W.FS_QSC)


@pytest.mark.parametrize("fb", ["1", "2"])
@pytest.mark.parametrize("separable", [True, False])
@pytest.mark.parametrize("op", [0, 1, 2, 3])
def test_box_qsc_fp64(rt, monkeypatch, fb, separable, op):
    """Quadratic short characteristics in 3D (downwind point mirrored into
    the next plane, linear last step) against the oracle, float64, every
    operator, both sweep block widths."""
    monkeypatch.setenv("RT_BOX_FB", fb)
    p = qsc_box(separable, nx=6, ny=7, nz=6, n_nu=5, kernel="r2", seed=11)
    h = rt.Handle(p, precision=rt.RT_P_FP64, max_restart=4)
    x = W.random_vectors(p.n, 1, 80 + op)[0]
    y = torch.empty(p.n, dtype=torch.float64, device="cuda:0")
    h.rt_apply(op, dev(x), y)
    torch.cuda.synchronize()
    ref = oracle_op(p, op, x)
    assert rel(y.cpu().numpy(), ref) < 1e-12
    assert np.abs(y.cpu().numpy() - ref).max() < 1e-12 * np.abs(ref).max()


def test_box_qsc_integer_offset_direction(rt):
    """Diagonal directions whose upwind and downwind points are exact cells,
    both sweep senses."""
    p = qsc_box(nx=6, ny=6, nz=6, spacing=(1.0, 1.0, 1.0))
    d = np.array([[1 / math.sqrt(2), 0.0, -1 / math.sqrt(2)], [0.0, -1 / math.sqrt(2), 1 / math.sqrt(2)]])
    p = dataclasses.replace(p, dirs=d, w_dir=np.array([0.5, 0.5]), P=np.ones((2, 2)))
    h = rt.Handle(p, precision=rt.RT_P_FP64, max_restart=8)
    x = W.random_vectors(p.n, 1, 91)[0]
    y = torch.empty(p.n, dtype=torch.float64, device="cuda:0")
    h.rt_apply(1, dev(x), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), O.lambda_op(p, x)) < 1e-13


@pytest.mark.parametrize("separable", [True, False])
@pytest.mark.parametrize("op", [0, 1])
def test_box_qsc_mixed(rt, separable, op):
    """The float32 quadratic sweep (series below an optical depth of 0.5)
    within the mixed-apply bar."""
    p = qsc_box(separable, nx=9, ny=8, nz=7, order=6, n_nu=8, kernel="r2", seed=12)
    h = rt.Handle(p, precision=rt.RT_P_MIXED, max_restart=8)
    x = W.random_vectors(p.n, 1, 95 + op, "uniform")[0]
    y = torch.empty(p.n, dtype=torch.float64, device="cuda:0")
    h.rt_apply(op, dev(x), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), oracle_op(p, op, x)) < 2e-5


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_box_qsc_solve(rt, prec):
    p = qsc_box(nx=6, ny=5, nz=6, order=4, n_nu=5, kernel="r2", eps=1e-3)
    xref = O.solve_gmres(p, tol=1e-14, restart=300, max_iter=600).x
    h = rt.Handle(p, precision=rt.RT_P_FP64 if prec == "fp64" else rt.RT_P_MIXED, max_restart=120)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda:0")
    info = h.rt_solve(None, x, tol=1e-13, tol_inner=1e-5, restart=120, max_outer=30)
    torch.cuda.synchronize()
    assert info["status"] == 0, info
    assert rel(x.cpu().numpy(), xref) < 1e-10


def lc_box(separable=True, **kw):
    p = small_box(**kw) if separable else nonseparable_box(**kw)
    return dataclasses.replace(p, formal_solver=W.FS_LC)


@pytest.mark.parametrize("separable", [True, False])
@pytest.mark.parametrize("op", [0, 1, 2, 3])
def test_box_lc_fp64(rt, separable, op):
    """Long characteristics (each point's ray traced back to the inflow plane)
    against the oracle, float64, every operator."""
    p = lc_box(separable, nx=6, ny=7, nz=6, n_nu=5, kernel="r2", seed=13)
    h = rt.Handle(p, precision=rt.RT_P_FP64, max_restart=4)
    x = W.random_vectors(p.n, 1, 100 + op)[0]
    y = torch.empty(p.n, dtype=torch.float64, device="cuda:0")
    h.rt_apply(op, dev(x), y)
    torch.cuda.synchronize()
    ref = oracle_op(p, op, x)
    assert rel(y.cpu().numpy(), ref) < 1e-12
    assert np.abs(y.cpu().numpy() - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("op", [0, 1])
def test_box_lc_mixed(rt, op):
    p = lc_box(False, nx=9, ny=8, nz=7, order=6, n_nu=8, kernel="r2", seed=14)
    h = rt.Handle(p, precision=rt.RT_P_MIXED, max_restart=8)
    x = W.random_vectors(p.n, 1, 110 + op, "uniform")[0]
    y = torch.empty(p.n, dtype=torch.float64, device="cuda:0")
    h.rt_apply(op, dev(x), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), oracle_op(p, op, x)) < 2e-5


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_box_lc_solve(rt, prec):
    p = lc_box(nx=6, ny=5, nz=6, order=4, n_nu=5, kernel="r2", eps=1e-3)
    xref = O.solve_gmres(p, tol=1e-14, restart=300, max_iter=600).x
    h = rt.Handle(p, precision=rt.RT_P_FP64 if prec == "fp64" else rt.RT_P_MIXED, max_restart=120)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda:0")
    info = h.rt_solve(None, x, tol=1e-13, tol_inner=1e-5, restart=120, max_outer=30)
    torch.cuda.synchronize()
    assert info["status"] == 0, info
    assert rel(x.cpu().numpy(), xref) < 1e-10


def test_long_characteristics_are_refused_for_columns(rt):
    col = W.two_level_column(np.logspace(-2, 2, 7), 4, 2, 5, "r2", 1e-3, 1.0, formal_solver=W.FS_LC)
    with pytest.raises(rt.RTError) as e:
        rt.Handle(col)
    assert e.value.code == rt.RT_ERR_ARG
