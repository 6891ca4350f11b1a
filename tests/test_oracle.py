"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each check is independent of the oracle's own formulas: closed forms,
alternative routes to the same quantity (closed-form matrix entries against
the recurrence, a reduced system against the full one), the sqrt(eps) law,
and the numbers printed in the paper.
"""
import dataclasses
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2602_21958_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# ------------------------------------------------------------- formal solvers
def test_w1_series_matches_closed_form_where_both_are_accurate():
    # w1/dtau = 1 - (1 - e^-d)/d; at d ~ 0.1 both branches are accurate to ~1e-15
    d = np.array([0.0999999, 0.1000001])
    ref = (d + np.expm1(-d)) / d
    assert np.allclose(O.w1_over_dtau(d), ref, rtol=1e-13, atol=0)
    # small-d limit: w1/d -> d/2
    assert abs(O.w1_over_dtau(np.array([1e-12]))[0] / 0.5e-12 - 1) < 1e-10


def test_scl_constant_source_closed_form():
    """S = B, no inflow: I = B (1 - e^{-tau}) exactly (products of e^-dtau telescope)."""
    p = W.config_c1()
    I = O.lambda_1d(p, 2.5 * np.ones(p.n)).reshape(p.nz, p.n_dir, p.n_nu)
    dt = O.dtau_1d(p)
    down = p.mu < 0
    tau_down = np.concatenate([np.zeros((1,) + dt.shape[1:]), np.cumsum(dt, axis=0)])
    tau_up = np.concatenate([np.cumsum(dt[::-1], axis=0)[::-1], np.zeros((1,) + dt.shape[1:])])
    assert np.abs(I[:, down] - 2.5 * (1 - np.exp(-tau_down[:, down]))).max() < 1e-14 * 2.5
    assert np.abs(I[:, ~down] - 2.5 * (1 - np.exp(-tau_up[:, ~down]))).max() < 1e-14 * 2.5


@pytest.mark.parametrize("fs,c,q", [(W.FS_SCL, 0.0, 0.0), (W.FS_SCL, 0.37, 0.0),
                                    (W.FS_QSC, 0.37, 0.0), (W.FS_QSC, 0.37, 0.011)])
def test_pure_absorption_rhs_closed_form(fs, c, q):
    """eps = 1 (no scattering): A = Id and I = b = Lambda t + I_in. With
    B = a + c t + q t^2, constant chi = phi(nu), zero inflow at the top and
    B(t_N) at the bottom, the formal-solution integral along each ray has a
    closed form (evaluated here in 40-digit arithmetic). SC-L integrates a
    source linear in optical depth exactly and QSC a quadratic one, except on
    the last step of a ray, which is linear. c = q = 0 is the textbook
    B (1 - e^{-tau/|mu|}). Separates the upwind, current and downwind weights
    of a step (a constant source only sees their sum) and checks both sweep
    senses."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    a = 1.3
    t = np.logspace(-3, np.log10(30.0), 48)
    p = W.two_level_column(t, 4, 1, 9, "crd", 1.0, a + c * t + q * t * t, formal_solver=fs)
    I = O.rhs(p).reshape(p.nz, p.n_dir, p.n_nu)
    small = dataclasses.replace(p, nz=6, z=t[:6], chi=p.chi[:6], gamma=p.gamma[:6], t_src=p.t_src[:6])
    assert np.array_equal(O.assemble_A(small), np.eye(small.n))
    B = lambda x: mp.mpf(a) + mp.mpf(c) * x + mp.mpf(q) * x * x
    ref = np.empty_like(I)
    for d, mu in enumerate(p.mu):
        sg = -1 if mu < 0 else 1            # t along the ray back from a point: t + sg s h
        for f in range(p.n_nu):
            h = abs(mu) / mp.mpf(p.chi[0, f])       # depth per unit optical depth along the ray
            for i, ti in enumerate(t):
                x = mp.mpf(ti)
                # S(t + sg s h) = s0 + s1 s + s2 s^2 in the ray's optical depth s
                s0, s1, s2 = B(x), sg * h * (mp.mpf(c) + 2 * mp.mpf(q) * x), mp.mpf(q) * h * h
                D = (x - mp.mpf(t[0])) / h if mu < 0 else (mp.mpf(t[-1]) - x) / h
                ed = mp.exp(-D)
                g0, g1, g2 = 1 - ed, 1 - (1 + D) * ed, 2 - (2 + 2 * D + D * D) * ed
                inflow = 0 if mu < 0 else B(mp.mpf(t[-1]))
                ref[i, d, f] = float(inflow * ed + s0 * g0 + s1 * g1 + s2 * g2)
    exact = np.ones(I.shape, dtype=bool)
    if q != 0.0:                            # linear last step of each QSC ray
        exact[-1, p.mu < 0] = False
        exact[0, p.mu > 0] = False
    assert np.abs(I - ref)[exact].max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(I - ref)[~exact].max(initial=0.0) <= 1e-2 * np.abs(ref).max()


@pytest.mark.parametrize("fs", [W.FS_SCL, W.FS_QSC])
def test_depth_dependent_opacity_constant_source(fs):
    """chi linear in depth: the optical depth of a step is the exact integral
    of chi (trapezoid rule exact), so a constant source with no inflow gives
    I = B (1 - e^{-tau/|mu|}), tau measured from the ray's entry point."""
    z = np.linspace(0.0, 6.0, 31) ** 1.5
    p = W.two_level_column(z, 4, 1, 5, "crd", 1.0, 1.0, formal_solver=fs)
    c0, c1 = 0.2, 0.9
    p = dataclasses.replace(p, chi=p.chi * (c0 + c1 * z)[:, None])
    B = 0.8
    I = O.lambda_op(p, np.full(p.n, B)).reshape(p.nz, p.n_dir, p.n_nu)
    col = c0 * z + 0.5 * c1 * z * z                     # int_0^z (c0 + c1 z') dz'
    phi = p.chi[0] / c0
    for d, mu in enumerate(p.mu):
        tau = (col if mu < 0 else col[-1] - col)[:, None] * phi[None, :] / abs(mu)
        assert np.abs(I[:, d] - B * -np.expm1(-tau)).max() <= 1e-14


def test_scl_inflow_equal_to_source_is_invariant():
    p = W.config_c1()
    I = O.lambda_1d(p, np.ones(p.n), with_inflow=True).reshape(p.nz, p.n_dir, p.n_nu)
    assert np.abs(I[:, p.mu > 0] - 1.0).max() < 1e-14


@pytest.mark.parametrize("du", [1e-6, 1e-3, 0.05, 0.0999, 0.1, 0.3, 1.0, 4.0, 30.0])
@pytest.mark.parametrize("ratio", [0.1, 1.0, 7.0])
def test_qsc_step_is_exact_for_quadratic_sources(du, ratio):
    # independent reference: adaptive quadrature of the formal-solution integral
    from scipy.integrate import quad
    dd = ratio * du
    e, pu, pc, pd = O.qsc_coefficients(np.array([du]), np.array([dd]))
    assert abs(e[0] - math.exp(-du)) <= 1e-15
    for p0, p1, p2 in ((1.0, 0.0, 0.0), (0.3, -1.7, 0.0), (0.2, 0.9, -2.3)):
        S = lambda s: p0 + p1 * s + p2 * s * s
        ref = quad(lambda s: S(s) * math.exp(-(du - s)), 0.0, du, epsabs=0.0, epsrel=2e-14, limit=200)[0]
        got = pu[0] * S(0.0) + pc[0] * S(du) + pd[0] * S(du + dd)
        scale = max(abs(p0), abs(p1) * du, abs(p2) * du * du) * -math.expm1(-du)
        assert abs(got - ref) <= 1e-12 * scale + 1e-300, (p0, p1, p2, got, ref)


def test_qsc_constant_source_closed_form():
    # S = B, zero inflow: I(tau) = B (1 - e^-tau) exactly along every ray
    t = np.logspace(-3, 3, 25)
    q = W.two_level_column(t, 4, 1, 5, "crd", 1.0, 1.0, formal_solver=W.FS_QSC)
    B = 1.7
    I = O.lambda_op(q, np.full(q.n, B)).reshape(q.nz, q.n_dir, q.n_nu)
    tau = np.concatenate([np.zeros((1, q.n_dir, q.n_nu)), np.cumsum(O.dtau_1d(q), axis=0)])
    down = q.mu < 0
    assert np.allclose(I[:, down], B * -np.expm1(-tau[:, down]), rtol=1e-13, atol=1e-15)


def test_qsc_converges_at_higher_order_than_scl():
    # smooth source along a constant-opacity slab: quadratic step error falls
    # faster under refinement than the linear one (exact integral as reference)
    errs = {}
    for fs in (W.FS_SCL, W.FS_QSC):
        e = []
        for nz in (41, 81, 161):
            t = np.linspace(0.0, 4.0, nz)
            q = W.two_level_column(t, 2, 1, 1, "crd", 1.0, 1.0, formal_solver=fs)
            tau_pts = np.cumsum(np.concatenate([[0.0], O.dtau_1d(q)[:, 0, 0]]))  # down ray 0
            src = np.sin(1.3 * tau_pts) + 2.0
            S = np.repeat(src[:, None], q.n_r, axis=1).ravel()
            I = O.lambda_op(q, S).reshape(nz, q.n_dir, q.n_nu)[:, 0, 0]
            mid = (nz - 1) // 2          # an interior point: every step before it is quadratic
            T = tau_pts[mid]
            ex = lambda s: (np.sin(1.3 * s) + 2.0) * np.exp(-(T - s))
            from scipy.integrate import quad
            ref = quad(ex, 0.0, T, epsabs=0, epsrel=1e-13, limit=400)[0]
            e.append(abs(I[mid] - ref))
        errs[fs] = e
    assert errs[W.FS_QSC][-1] < errs[W.FS_SCL][-1] / 10
    assert errs[W.FS_QSC][1] / errs[W.FS_QSC][2] > 6.0   # about third order


def test_ie_recurrence_equals_closed_form_entries():
    """Dense Lambda from the recurrence (eqs. ie_1, ie_2) equals the closed-form
    entries of eqs. ie_mono3, ie_mono4, including the zero first row of
    Lambda_down and zero last row of Lambda_up."""
    q = W.paper_iso(7, 3, "crd")
    L1 = O.lambda_matrix_1d(q)
    L2 = O.lambda_ie_closed_form(q)
    assert np.abs(L1 - L2).max() < 1e-15
    nr = q.n_r
    for d in range(q.n_dir):
        for f in range(q.n_nu):
            idx = np.arange(q.nz) * nr + d * q.n_nu + f
            blk = L1[np.ix_(idx, idx)]
            if q.mu[d] < 0:
                assert np.all(blk[0] == 0) and np.allclose(blk, np.tril(blk))
            else:
                assert np.all(blk[-1] == 0) and np.allclose(blk, np.triu(blk))


def test_ie_uniform_grid_entries():
    """Thm main3: on a uniform grid the entries are dtau/(1+dtau)^(i-j+1)."""
    q = W.paper_mono(9, 2)
    L = O.lambda_matrix_1d(q)
    d = q.n_dir
    for k in range(d):
        dtau = (q.z[1] - q.z[0]) / abs(q.mu[k])
        idx = np.arange(q.nz) * q.n_r + k
        blk = L[np.ix_(idx, idx)]
        for i in range(q.nz):
            for j in range(q.nz):
                if q.mu[k] < 0 and 1 <= j <= i:
                    ref = dtau / (1 + dtau) ** (i - j + 1)
                elif q.mu[k] > 0 and i <= j <= q.nz - 2:
                    ref = dtau / (1 + dtau) ** (j - i + 1)
                else:
                    ref = 0.0
                assert abs(blk[i, j] - ref) < 1e-15


def test_lambda_block_diagonal_in_rays():
    q = W.paper_iso(5, 3, "coherent")
    L = O.lambda_matrix_1d(q)
    nr = q.n_r
    for a in range(q.n):
        for b in np.nonzero(L[a])[0]:
            assert a % nr == b % nr


# ------------------------------------------------------------------ scattering
def test_legendre_kernel_rank_and_symmetry():
    q = W.paper_mono(4, 24)
    psi = q.P
    assert np.allclose(psi, psi.T, atol=0)
    s = np.linalg.svd(psi, compute_uv=False)
    assert int(np.sum(s > 1e-10 * s[0])) == 8  # L + 1 (Sec. 5.1)


def test_sigma_matches_assembled_block_diagonal():
    q = W.paper_iso(4, 5, "crd")
    x = np.random.default_rng(1).standard_normal(q.n)
    assert np.allclose(O.sigma_matrix(q) @ x, O.sigma_op(q, x), rtol=1e-14, atol=1e-14)


def test_dense_kernel_equals_separable_kernel():
    """Psi = P (x) R (the dense form, eq. Sigma) must give the factored
    contraction's result, with non-uniform direction and frequency weights
    (dipole x R_II-A, two azimuths)."""
    q = W.two_level_column(np.logspace(-2, 2, 3), 4, 2, 6, "r2", 1e-2, 1.0)
    dq = q.with_dense_kernel()
    x = np.random.default_rng(2).standard_normal(q.n)
    ref = O.sigma_op(q, x)
    assert np.abs(O.sigma_op(dq, x) - ref).max() <= 1e-14 * np.abs(ref).max()
    assert np.abs(O.sigma_matrix(dq) @ x - ref).max() <= 1e-14 * np.abs(ref).max()


def test_crd_reduces_to_mean_intensity():
    """Isotropic CRD: S = (1 - eps) Jbar + eps B, Jbar = sum w w phi I."""
    p = W.config_c1()
    x = np.random.default_rng(2).uniform(size=p.n)
    S = O.sigma_op(p, x, with_source=True).reshape(p.nz, p.n_dir, p.n_nu)
    _, wn, phi, _ = W.line_data(21, "crd")
    X = x.reshape(p.nz, p.n_dir, p.n_nu)
    J = np.einsum("idn,d,n->i", X, p.w_dir, wn * phi)
    ref = (1 - 1e-4) * J + 1e-4
    assert np.abs(S - ref[:, None, None]).max() < 1e-14


def test_dipole_scattering_conserves_photons():
    """sum_Omega' w P(Omega, Omega') = 1 for the dipole phase with GL (azimuth
    averaged) and level-symmetric (3D) sets; with conservative R the whole
    kernel returns phi(nu)."""
    d, w = W.gauss_legendre_directions(8, 2)
    assert np.allclose(W.dipole_azimuth_averaged(d[:, 2]) @ w, 1.0, atol=1e-15)
    for order in (6, 8):
        d, w = W.level_symmetric(order)
        assert np.allclose(W.dipole_3d(d) @ w, 1.0, atol=1e-14)
    x, wn, phi, R = W.line_data(64, "r2")
    assert np.allclose(R @ wn, phi, rtol=1e-13)
    assert np.allclose(R, R.T, atol=1e-16)


# --------------------------------------------------------------- global system
def test_matrix_free_apply_equals_assembled():
    for q in (W.paper_iso(6, 5, "crd"), W.paper_mono(8, 6),
              dataclasses.replace(W.two_level_column(np.logspace(-2, 2, 7), 4, 2, 9, "r2", 1e-2, 1.0),
                                  formal_solver=W.FS_SCL)):
        A = O.assemble_A(q)
        for seed in range(2):
            x = np.random.default_rng(seed).standard_normal(q.n)
            ref = A @ x
            assert np.linalg.norm(O.apply_A(q, x) - ref) <= 1e-14 * np.linalg.norm(ref)


def test_lu_equals_gmres():
    q = W.two_level_column(np.logspace(-3, 3, 12), 4, 2, 7, "r2", 1e-3, 1.0)
    x_lu = O.solve_dense(q)
    g = O.solve_gmres(q, tol=1e-14, restart=400, max_iter=400)
    assert np.linalg.norm(g.x - x_lu) <= 1e-12 * np.linalg.norm(x_lu)


def test_restarted_gmres_cycles_minimise_the_residual():
    """Each GMRES(m) cycle returns the minimiser of ||b - A x|| over
    x_prev + K_m(A, r_prev) (the method's definition): two cycles of m = 3
    against least squares on explicit Krylov bases."""
    rng = np.random.default_rng(13)
    n, m = 30, 3
    A = np.eye(n) + 0.5 * rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    x = np.zeros(n)
    for _ in range(2):
        r = b - A @ x
        K = np.stack([np.linalg.matrix_power(A, k) @ r for k in range(m)], axis=1)
        y = np.linalg.lstsq(A @ K, r, rcond=None)[0]
        x = x + K @ y
    got = O.gmres(lambda v: A @ v, b, tol=1e-300, restart=m, max_iter=2 * m)
    assert got.restarts == 2 and got.iterations == 2 * m
    assert np.abs(got.x - x).max() <= 1e-12 * np.abs(x).max()


def test_bicgstab_solves_a_random_nonsymmetric_system():
    # library LU as the independent reference; a wrong beta/omega or sign stalls
    rng = np.random.default_rng(7)
    A = np.eye(60) + 0.3 * rng.standard_normal((60, 60)) / np.sqrt(60)
    b = rng.standard_normal(60)
    r = O.bicgstab(lambda v: A @ v, b, tol=1e-14)
    x = np.linalg.solve(A, b)
    assert r.relres <= 1e-13
    assert np.linalg.norm(r.x - x) <= 1e-12 * np.linalg.norm(x)


def test_bicgstab_on_a_multiple_of_identity_takes_one_half_step():
    b = np.random.default_rng(8).standard_normal(30)
    r = O.bicgstab(lambda v: 2.5 * v, b, tol=1e-14)
    assert r.iterations == 1
    assert np.allclose(r.x, b / 2.5, rtol=0, atol=1e-15)


def test_bicgstab_terminates_after_as_many_iterations_as_distinct_eigenvalues():
    """The BiCG polynomial of BiCGStab annihilates r0 once its degree reaches
    that of the minimal polynomial of A with respect to r0: a diagonalisable
    non-normal A with 3 distinct eigenvalues is solved in at most 3
    iterations (any error in the direction recurrence loses this)."""
    rng = np.random.default_rng(9)
    n = 40
    lam = np.repeat([1.0, 2.0, 3.5], [15, 15, 10])
    X = np.eye(n) + 0.2 * rng.standard_normal((n, n)) / np.sqrt(n)
    A = X @ np.diag(lam) @ np.linalg.inv(X)
    b = rng.standard_normal(n)
    r = O.bicgstab(lambda v: A @ v, b, tol=1e-11)
    assert r.iterations <= 3 and r.relres <= 1e-11


def test_bicgstab_first_iteration_is_galerkin_then_minimal_residual():
    """x0 = 0: the first iterate is x1 = alpha b + omega s with s = b - alpha A b,
    alpha fixed by the Petrov-Galerkin condition (b, s) = 0 and omega by the
    least-squares problem min ||s - omega A s|| (solved here by lstsq)."""
    rng = np.random.default_rng(10)
    A = np.eye(25) + 0.4 * rng.standard_normal((25, 25)) / 5.0
    b = rng.standard_normal(25)
    x1 = O.bicgstab(lambda v: A @ v, b, tol=1e-300, max_iter=1).x
    # alpha: the root of (b, b - alpha A b) = 0, found by lstsq on the 1x1 system
    alpha = np.linalg.lstsq((b @ A @ b).reshape(1, 1), np.array([b @ b]), rcond=None)[0][0]
    s = b - alpha * (A @ b)
    omega = np.linalg.lstsq((A @ s).reshape(-1, 1), s, rcond=None)[0][0]
    assert np.abs(x1 - (alpha * b + omega * s)).max() <= 1e-13 * np.abs(x1).max()


def test_lu_equals_bicgstab():
    q = W.two_level_column(np.logspace(-3, 3, 12), 4, 2, 7, "r2", 1e-3, 1.0)
    x_lu = O.solve_dense(q)
    r = O.solve_bicgstab(q, tol=1e-14)
    assert np.linalg.norm(r.x - x_lu) <= 1e-11 * np.linalg.norm(x_lu)


def test_arnoldi_full_space_gives_the_eigenvalues():
    # library eigenvalues as the independent reference; Arnoldi relation A V = V H
    rng = np.random.default_rng(9)
    A = np.eye(40) + 0.4 * rng.standard_normal((40, 40)) / np.sqrt(40)
    H = O.arnoldi(lambda v: A @ v, rng.standard_normal(40), 40)
    assert H.shape == (41, 40)
    ritz = np.sort_complex(np.linalg.eigvals(H[:40, :40]))
    lam = np.sort_complex(np.linalg.eigvals(A))
    assert np.abs(ritz - lam).max() < 1e-9
    assert np.allclose(np.tril(H, -2), 0.0)


def test_arnoldi_ritz_values_reproduce_table_mono():
    # full Arnoldi on the Sec. 5.1 operator: the Ritz values are the spectrum,
    # so the printed cluster fraction (Table mono) comes back
    p = W.paper_mono(10, 12)
    H = O.arnoldi(lambda v: O.apply_A(p, v), np.ones(p.n), p.n)
    k = H.shape[1]
    ritz = np.linalg.eigvals(H[:k, :k])
    lam = np.linalg.eigvals(O.assemble_A(p))
    frac = lambda z: np.mean((np.abs(z) >= 0.999) & (np.abs(z) <= 1 + 1e-12))
    if k == p.n:
        assert abs(frac(ritz) - frac(lam)) < 1e-12
    # a Krylov space that became invariant early holds exact eigenvalues
    d = np.abs(ritz[:, None] - lam[None, :]).min(axis=1)
    assert d.max() < 1e-8


def test_reduced_crd_system_equals_full_solve():
    """Independent route at full C1 size: the N_z x N_z reduced CRD system."""
    p = W.config_c1()
    g = O.solve_gmres(p, tol=1e-14, restart=200, max_iter=400)
    Ir = O.solve_crd_reduced(p)
    assert np.linalg.norm(Ir - g.x) <= 1e-12 * np.linalg.norm(Ir)


def test_sqrt_eps_law():
    """Semi-infinite isothermal CRD atmosphere: S(0) = sqrt(eps) B.  The
    discrete value converges to it at first order in points per decade."""
    errs = []
    eps = 1e-4
    _, wn, phi, _ = W.line_data(21, "crd")
    for n in (60, 120, 240):
        t = np.logspace(-6, 8, n)
        q = W.two_level_column(t, 8, 1, 21, "crd", eps, 1.0)
        I = O.solve_crd_reduced(q).reshape(q.nz, q.n_dir, q.n_nu)
        J = np.einsum("dn,d,n->", I[0], q.w_dir, wn * phi)
        S0 = (1 - eps) * J + eps
        errs.append(abs(S0 / math.sqrt(eps) - 1.0))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.15
    assert 0.3 < errs[2] / errs[1] < 0.7


# ------------------------------------------------------------ paper's numbers
_MONO_MISMATCH = pytest.mark.xfail(strict=True, reason="printed entry not reproduced (N_Omega = 50 column "
                                   "and (40, 24)); no neighbouring N_Omega reproduces it either")


@pytest.mark.parametrize("n_s,n_omega", [(10, 12), (10, 24), (20, 12), (20, 24), (40, 12), (10, 100),
                                         (20, 100), (40, 100), (100, 12), (100, 24), (200, 12),
                                         pytest.param(10, 50, marks=_MONO_MISMATCH),
                                         pytest.param(20, 50, marks=_MONO_MISMATCH),
                                         pytest.param(40, 50, marks=_MONO_MISMATCH),
                                         pytest.param(100, 50, marks=_MONO_MISMATCH),
                                         pytest.param(40, 24, marks=_MONO_MISMATCH)])
def test_table_mono(n_s, n_omega):
    tab = GOLDEN["table_mono"]
    ref = tab["rows"][str(n_s)][tab["n_omega"].index(n_omega)]
    frac, lmin = O.cluster_fraction(O.assemble_A(W.paper_mono(n_s, n_omega)))
    assert abs(100 * frac - ref) <= 0.05 + 1e-9
    # Sec. 5.1 states |lambda|_min > 0.82.  The oracle meets it strictly up to
    # N_s = 20 (0.82037-0.82186); from N_s = 40 on its smallest modulus sits
    # just below (0.81920-0.81972, decreasing with N_s), a documented
    # deviation of less than 1e-3 that is asserted as such, not rounded away.
    if n_s <= 20:
        assert lmin > tab["abs_lambda_min_gt"]
    else:
        assert 0.8190 < lmin < tab["abs_lambda_min_gt"]


@pytest.mark.parametrize("n", [10, 50])
def test_gmres_iso_coherent_iteration_counts(n):
    ref = GOLDEN["gmres_iso_coherent"]["n_to_iterations"][str(n)]
    q = W.paper_iso(n, n, "coherent", n_mu=n)
    r = O.gmres(lambda v: O.apply_A(q, v), np.ones(q.n), tol=1e-15, restart=200, max_iter=60)
    first = next(i for i, h in enumerate(r.history) if h < 1e-15 * 10)
    assert first == ref


@pytest.mark.parametrize("n_s,n_nu", [(10, 10), (10, 20), (20, 10)])
def test_iso_crd_cluster_and_lower_bound(n_s, n_nu):
    frac, lmin = O.cluster_fraction(O.assemble_A(W.paper_iso(n_s, n_nu, "crd")))
    assert 100 * frac > GOLDEN["table_iso"]["crd_all_gt"]
    assert lmin > GOLDEN["table_iso"]["abs_lambda_min_gt"]
    frac_c, lmin_c = O.cluster_fraction(O.assemble_A(W.paper_iso(n_s, n_nu, "coherent")))
    assert lmin_c > GOLDEN["table_iso"]["abs_lambda_min_gt"]


def test_cluster_fraction_counts_the_band():
    """|lambda| in [0.999, 1 + 1e-12] (Tables mono and iso), on a non-normal
    matrix with known eigenvalues: 0.9995 and 1 count; 1.0005, 1.5, 0.5 do not."""
    rng = np.random.default_rng(11)
    lam = np.array([0.9995, 1.0, 1.0005, 1.5, 0.5, 1.0, 0.9985, 0.9991])
    X = np.eye(8) + 0.1 * rng.standard_normal((8, 8))
    frac, lmin = O.cluster_fraction(X @ np.diag(lam) @ np.linalg.inv(X))
    assert frac == 4 / 8
    assert abs(lmin - 0.5) < 1e-12


def test_cluster_fraction_grows_under_refinement():
    """Thm main4: the fraction in D(1, 1e-3) does not decrease as N_s, N_Omega grow."""
    f = [O.cluster_fraction(O.assemble_A(W.paper_mono(ns, 12)))[0] for ns in (10, 20, 40)]
    assert f[0] <= f[1] <= f[2]
    g = [O.cluster_fraction(O.assemble_A(W.paper_mono(10, no)))[0] for no in (12, 24)]
    assert g[0] <= g[1]


# ------------------------------------------------------------------ 3D transfer
def _homogeneous_box(n, nz, chi_z, dirs, w):
    nn = 2
    npts = n * n * nz
    chi = np.repeat(chi_z[:, None], n * n, axis=1).reshape(npts, 1) * np.array([[1.0, 0.3]])
    return W.Problem(dims=3, nx=n, ny=n, nz=nz, z=np.array([1.0, 1.0, 1.0]), dirs=dirs,
                     w_dir=w, w_nu=np.ones(nn) / nn, chi=chi, gamma=np.zeros((npts, nn)),
                     P=np.ones((len(w), len(w))), R=np.ones((nn, nn)), I_top=np.zeros(nn),
                     I_bot=np.ones(nn), formal_solver=W.FS_SCL)


def test_3d_homogeneous_box_reduces_to_1d_columns():
    """chi and S uniform in x, y: bilinear interpolation is exact, so every
    column equals the 1D solution with mu = Omega_z."""
    rng = np.random.default_rng(3)
    nz, n = 9, 5
    dirs, w = W.level_symmetric(6)
    chi_z = rng.uniform(0.2, 2.0, nz)
    box = _homogeneous_box(n, nz, chi_z, dirs, w)
    Sz = rng.standard_normal((nz, 1, 1, len(w), 2))
    S = np.broadcast_to(Sz, (nz, n, n, len(w), 2)).reshape(-1)
    I3 = O.lambda_3d(box, S, with_inflow=True).reshape(nz, n, n, len(w), 2)
    col = W.Problem(dims=1, nx=1, ny=1, nz=nz, z=np.arange(nz, dtype=float), dirs=dirs, w_dir=w,
                    w_nu=box.w_nu, chi=chi_z[:, None] * np.array([[1.0, 0.3]]),
                    gamma=np.zeros((nz, 2)), I_top=box.I_top, I_bot=box.I_bot)
    I1 = O.lambda_1d(col, Sz.reshape(-1), with_inflow=True).reshape(nz, len(w), 2)
    assert np.abs(I3 - I1[:, None, None]).max() < 1e-14


def test_3d_integer_offset_follows_the_diagonal():
    """Omega = (1, 0, -1)/sqrt(2), unit cells: the upwind point is exactly the
    cell (x-1, y, k-1), so each diagonal line is an independent 1D ray."""
    rng = np.random.default_rng(4)
    n, nz = 6, 5
    dirs = np.array([[1 / math.sqrt(2), 0.0, -1 / math.sqrt(2)]])
    box = W.Problem(dims=3, nx=n, ny=n, nz=nz, z=np.array([1.0, 1.0, 1.0]), dirs=dirs,
                    w_dir=np.ones(1), w_nu=np.ones(1), chi=rng.uniform(0.1, 3, (n * n * nz, 1)),
                    gamma=np.zeros((n * n * nz, 1)), I_top=np.zeros(1), I_bot=np.zeros(1))
    S = rng.standard_normal(box.n)
    I = O.lambda_3d(box, S).reshape(nz, n, n)
    Sg = S.reshape(nz, n, n)
    chi = box.chi.reshape(nz, n, n)
    ds = math.sqrt(2.0)
    for y in range(n):
        for x0 in range(n):
            val = 0.0
            for k in range(1, nz):
                xu, xc = (x0 + k - 1) % n, (x0 + k) % n
                d = 0.5 * (chi[k - 1, y, xu] + chi[k, y, xc]) * ds
                e = math.exp(-d)
                beta = (d + math.expm1(-d)) / d
                val = e * val + (1 - e - beta) * Sg[k - 1, y, xu] + beta * Sg[k, y, xc]
                assert abs(I[k, y, xc] - val) < 1e-13
            assert I[0, y, x0] == 0.0


def _diagonal_qsc(chi_line, S_line, ds):
    """1D quadratic short characteristics along one ray through the cells
    chi_line[k], S_line[k] (k in sweep order, unit segments of length ds): the
    upwind, current and downwind cells of step k are k-1, k, k+1; the last
    step is linear.  Inflow 0."""
    nz = len(S_line)
    out = np.zeros(nz)
    for k in range(1, nz):
        du = 0.5 * (chi_line[k - 1] + chi_line[k]) * ds
        if k < nz - 1:
            dd = 0.5 * (chi_line[k] + chi_line[k + 1]) * ds
            e, pu, pc, pd = O.qsc_coefficients(np.array(du), np.array(dd))
            src = pu * S_line[k - 1] + pc * S_line[k] + pd * S_line[k + 1]
        else:
            e, al, be = O.step_coefficients(np.array(du), W.FS_SCL)
            src = al * S_line[k - 1] + be * S_line[k]
        out[k] = e * out[k - 1] + src
    return out


@pytest.mark.parametrize("sgn", [-1.0, 1.0])
def test_3d_qsc_integer_offset_follows_the_diagonal(sgn):
    """Quadratic short characteristics in 3D with Omega = (1, 0, sgn)/sqrt(2),
    unit cells: upwind and downwind points are exactly the cells (x -+ 1) of
    the neighbouring planes, so every diagonal line is an independent 1D QSC
    ray (a downwind shift taken with the wrong sign, or a wrong downwind
    plane, breaks it)."""
    rng = np.random.default_rng(14)
    n, nz = 6, 7
    dirs = np.array([[1 / math.sqrt(2), 0.0, sgn / math.sqrt(2)]])
    box = W.Problem(dims=3, nx=n, ny=n, nz=nz, z=np.array([1.0, 1.0, 1.0]), dirs=dirs,
                    w_dir=np.ones(1), w_nu=np.ones(1), chi=rng.uniform(0.05, 3, (n * n * nz, 1)),
                    gamma=np.zeros((n * n * nz, 1)), I_top=np.zeros(1), I_bot=np.zeros(1),
                    formal_solver=W.FS_QSC)
    S = rng.standard_normal(box.n)
    I = O.lambda_3d(box, S).reshape(nz, n, n)
    Sg = S.reshape(nz, n, n)
    chi = box.chi.reshape(nz, n, n)
    planes = list(range(nz)) if sgn < 0 else list(range(nz - 1, -1, -1))  # sweep order
    for y in range(n):
        for x0 in range(n):
            xs = [(x0 + i) % n for i in range(nz)]         # the ray moves +1 in x per plane
            ref = _diagonal_qsc(np.array([chi[k, y, x] for k, x in zip(planes, xs)]),
                                np.array([Sg[k, y, x] for k, x in zip(planes, xs)]), math.sqrt(2.0))
            got = np.array([I[k, y, x] for k, x in zip(planes, xs)])
            assert np.abs(got - ref).max() < 1e-13


def test_3d_qsc_homogeneous_box_is_the_1d_column():
    """A box whose opacity and source vary only with z: with QSC every
    direction of every cell reproduces the 1D QSC column (Sec. 3.2 recurrence
    with the quadratic integrator) for mu = Omega_z, with inflow."""
    rng = np.random.default_rng(15)
    nx, ny, nz, nn = 4, 3, 8, 3
    dirs, wd = W.level_symmetric(4)
    chi1 = rng.uniform(0.05, 4.0, (nz, nn))
    S1 = rng.standard_normal((nz, len(dirs), nn))
    dz = 0.7
    box = W.Problem(dims=3, nx=nx, ny=ny, nz=nz, z=np.array([1.1, 0.9, dz]), dirs=dirs, w_dir=wd,
                    w_nu=np.ones(nn), chi=np.repeat(chi1, nx * ny, axis=0),
                    gamma=np.zeros((nx * ny * nz, nn)), I_top=rng.uniform(0, 1, nn),
                    I_bot=rng.uniform(0, 1, nn), formal_solver=W.FS_QSC)
    col = W.Problem(dims=1, nx=1, ny=1, nz=nz, z=dz * np.arange(nz), dirs=dirs, w_dir=wd,
                    w_nu=np.ones(nn), chi=chi1, gamma=np.zeros((nz, nn)), I_top=box.I_top,
                    I_bot=box.I_bot, formal_solver=W.FS_QSC)
    S3 = np.broadcast_to(S1[:, None, None], (nz, ny, nx, len(dirs), nn)).reshape(-1)
    I3 = O.lambda_3d(box, S3, with_inflow=True).reshape(nz, ny, nx, len(dirs), nn)
    I1 = O.lambda_op(col, S1.reshape(-1), with_inflow=True).reshape(nz, len(dirs), nn)
    assert np.abs(I3 - I1[:, None, None]).max() < 1e-13 * np.abs(I1).max()


def _lc_box(rng, dirs, n=(5, 4, 6), nn=2, fs=None):
    nx, ny, nz = n
    return W.Problem(dims=3, nx=nx, ny=ny, nz=nz, z=np.array([1.0, 1.3, 0.8]), dirs=dirs,
                     w_dir=np.ones(len(dirs)) / len(dirs), w_nu=np.ones(nn),
                     chi=rng.uniform(0.05, 3.0, (nx * ny * nz, nn)), gamma=np.zeros((nx * ny * nz, nn)),
                     I_top=rng.uniform(0, 1, nn), I_bot=rng.uniform(0, 1, nn),
                     formal_solver=fs or W.FS_LC)


def test_3d_lc_integer_offsets_equal_short_characteristics():
    """With integer cell offsets per plane the ray of every point passes
    through cell centres only, so long characteristics and the SC-L plane
    sweep compute the same recurrence (both senses, with inflow)."""
    rng = np.random.default_rng(21)
    # with dx = 1, dy = 1.3, dz = 0.8: Omega ~ (1, 1.3, -0.8) moves (1, 1) cells per
    # plane downwards, Omega ~ (-1, 0, 0.8) moves (-1, 0) cells per plane upwards
    dirs = np.array([[1.0, 1.3, -0.8], [-1.0, 0.0, 0.8]])
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    box = _lc_box(rng, dirs)
    S = rng.standard_normal(box.n)
    lc = O.lambda_op(box, S, with_inflow=True)
    sc = O.lambda_op(dataclasses.replace(box, formal_solver=W.FS_SCL), S, with_inflow=True)
    assert np.abs(lc - sc).max() < 1e-13 * np.abs(sc).max()


def test_3d_lc_homogeneous_box_is_the_1d_column():
    """Fields that vary only with z: every long characteristic sees the 1D
    column, whatever the horizontal offsets (level-symmetric S_4)."""
    rng = np.random.default_rng(22)
    nx, ny, nz, nn = 4, 3, 7, 2
    dirs, wd = W.level_symmetric(4)
    chi1 = rng.uniform(0.05, 4.0, (nz, nn))
    S1 = rng.standard_normal((nz, len(dirs), nn))
    box = W.Problem(dims=3, nx=nx, ny=ny, nz=nz, z=np.array([1.1, 0.9, 0.7]), dirs=dirs, w_dir=wd,
                    w_nu=np.ones(nn), chi=np.repeat(chi1, nx * ny, axis=0), gamma=np.zeros((nx * ny * nz, nn)),
                    I_top=rng.uniform(0, 1, nn), I_bot=rng.uniform(0, 1, nn), formal_solver=W.FS_LC)
    col = W.Problem(dims=1, nx=1, ny=1, nz=nz, z=0.7 * np.arange(nz), dirs=dirs, w_dir=wd, w_nu=np.ones(nn),
                    chi=chi1, gamma=np.zeros((nz, nn)), I_top=box.I_top, I_bot=box.I_bot)
    S3 = np.broadcast_to(S1[:, None, None], (nz, ny, nx, len(dirs), nn)).reshape(-1)
    I3 = O.lambda_op(box, S3, with_inflow=True).reshape(nz, ny, nx, len(dirs), nn)
    I1 = O.lambda_op(col, S1.reshape(-1), with_inflow=True).reshape(nz, len(dirs), nn)
    assert np.abs(I3 - I1[:, None, None]).max() < 1e-13 * np.abs(I1).max()


def test_3d_lc_single_rays_by_hand():
    """Fractional offsets: a few points recomputed one scalar at a time (the
    ray's crossing of every plane, bilinear weights from the floor and the
    fraction of the offset, periodic wrap), and the long characteristics
    differ from the short ones there (the intensity is not interpolated)."""
    rng = np.random.default_rng(23)
    v = np.array([[0.37, -0.52, -0.6], [-0.21, 0.44, 0.7]])
    dirs = v / np.linalg.norm(v, axis=1)[:, None]
    box = _lc_box(rng, dirs, n=(5, 4, 6), nn=1)
    nx, ny, nz = box.nx, box.ny, box.nz
    S = rng.standard_normal(box.n)
    I = O.lambda_op(box, S, with_inflow=True).reshape(nz, ny, nx, 2)
    Sg = S.reshape(nz, ny, nx, 2)
    chi = box.chi.reshape(nz, ny, nx)
    dx, dy, dz = box.z

    def interp(F, k, yy, xx, sx, sy):
        px, py = xx - sx, yy - sy
        x0, y0 = math.floor(px), math.floor(py)
        ax, ay = px - x0, py - y0
        g = lambda j, i: F[k, j % ny, i % nx]
        return ((1 - ay) * ((1 - ax) * g(y0, x0) + ax * g(y0, x0 + 1))
                + ay * ((1 - ax) * g(y0 + 1, x0) + ax * g(y0 + 1, x0 + 1)))

    for d in range(2):
        ox, oy, oz = dirs[d]
        ds = dz / abs(oz)
        sx, sy = ox * ds / dx, oy * ds / dy
        first, step = (nz - 1, -1) if oz > 0 else (0, 1)
        inflow = box.I_bot[0] if oz > 0 else box.I_top[0]
        for (k, yy, xx) in ((first + 5 * step, 1, 2), (first + 3 * step, 3, 0), (first + 1 * step, 0, 4)):
            s = abs(k - first)
            val, Sa, ca = inflow, None, None
            for m in range(s + 1):
                km, t = first + m * step, s - m
                Sm = interp(Sg[..., d], km, yy, xx, t * sx, t * sy)
                cm = interp(chi, km, yy, xx, t * sx, t * sy)
                if m > 0:
                    tau = 0.5 * (ca + cm) * ds
                    e = math.exp(-tau)
                    beta = (tau + math.expm1(-tau)) / tau
                    val = e * val + (1 - e - beta) * Sa + beta * Sm
                Sa, ca = Sm, cm
            assert abs(I[k, yy, xx, d] - val) < 1e-13 * max(1.0, abs(val))
    sc = O.lambda_op(dataclasses.replace(box, formal_solver=W.FS_SCL), S, with_inflow=True)
    assert np.abs(sc.reshape(I.shape) - I).max() > 1e-3


def test_3d_half_offset_interpolates_two_cells():
    """Upwind offset of half a cell in y: the upwind value is the mean of the
    two neighbouring cells of the upwind plane."""
    rng = np.random.default_rng(5)
    n, nz = 4, 2
    oy, oz = 0.5, 1.0
    nrm = math.hypot(oy, oz)
    dirs = np.array([[0.0, oy / nrm, oz / nrm]])  # upward, upwind plane k+1
    box = W.Problem(dims=3, nx=n, ny=n, nz=nz, z=np.array([1.0, 1.0, 1.0]), dirs=dirs,
                    w_dir=np.ones(1), w_nu=np.ones(1), chi=np.ones((n * n * nz, 1)),
                    gamma=np.zeros((n * n * nz, 1)), I_top=np.zeros(1), I_bot=np.zeros(1))
    S = rng.standard_normal(box.n)
    I = O.lambda_3d(box, S).reshape(nz, n, n)
    Sg = S.reshape(nz, n, n)
    d = 1.0 / dirs[0, 2]
    e = math.exp(-d)
    beta = (d + math.expm1(-d)) / d
    for y in range(n):
        for x in range(n):
            su = 0.5 * (Sg[1, (y - 1) % n, x] + Sg[1, y, x])
            ref = (1 - e - beta) * su + beta * Sg[0, y, x]
            assert abs(I[0, y, x] - ref) < 1e-14


def test_3d_fractional_offset_bilinear_upwind_point():
    """Upwind offset (0.3, 0.6) cells: I, S and chi at the upwind point are
    the bilinear blends of the four surrounding cells of the upwind plane
    (weights 0.7/0.3 in x, 0.4/0.6 in y), periodic in x and y."""
    rng = np.random.default_rng(6)
    n, nz = 5, 3
    ox, oy, oz = 0.3, 0.6, -1.0                 # downward: upwind plane k-1
    nrm = math.sqrt(ox * ox + oy * oy + oz * oz)
    dirs = np.array([[ox / nrm, oy / nrm, oz / nrm]])
    box = W.Problem(dims=3, nx=n, ny=n, nz=nz, z=np.array([1.0, 1.0, 1.0]), dirs=dirs,
                    w_dir=np.ones(1), w_nu=np.ones(1), chi=rng.uniform(0.2, 2.0, (n * n * nz, 1)),
                    gamma=np.zeros((n * n * nz, 1)), I_top=np.zeros(1), I_bot=np.zeros(1))
    S = rng.standard_normal(box.n)
    I = O.lambda_3d(box, S).reshape(nz, n, n)
    Sg = S.reshape(nz, n, n)
    chi = box.chi.reshape(nz, n, n)
    ds = 1.0 / abs(dirs[0, 2])                  # path length between planes (dz = 1)

    def upwind(F, y, x):                        # F at (x - 0.3, y - 0.6)
        return (0.4 * (0.7 * F[y, x] + 0.3 * F[y, (x - 1) % n])
                + 0.6 * (0.7 * F[(y - 1) % n, x] + 0.3 * F[(y - 1) % n, (x - 1) % n]))

    for k in range(1, nz):
        for y in range(n):
            for x in range(n):
                d = 0.5 * (upwind(chi[k - 1], y, x) + chi[k, y, x]) * ds
                e = math.exp(-d)
                beta = (d + math.expm1(-d)) / d
                ref = (e * upwind(I[k - 1], y, x) + (1 - e - beta) * upwind(Sg[k - 1], y, x)
                       + beta * Sg[k, y, x])
                assert abs(I[k, y, x] - ref) < 1e-13


def test_3d_constant_source_closed_form():
    n, nz = 4, 6
    dirs, w = W.level_symmetric(4)
    box = _homogeneous_box(n, nz, np.full(nz, 0.7), dirs, w)
    I = O.lambda_3d(box, np.ones(box.n)).reshape(nz, n * n, len(w), 2)
    for d in range(len(w)):
        ds = 1.0 / abs(dirs[d, 2])
        for f, c in enumerate((0.7, 0.21)):
            steps = np.arange(nz) if dirs[d, 2] < 0 else np.arange(nz)[::-1]
            ref = 1 - np.exp(-c * ds * steps)
            assert np.abs(I[:, :, d, f] - ref[:, None]).max() < 1e-14


# ------------------------------------------------------------------ batches
def _ragged_columns():
    return [W.two_level_column(np.logspace(-2, 2, 5), 4, 1, 3, "crd", 1e-2, 1.0),
            W.two_level_column(np.logspace(-3, 3, 9), 2, 2, 7, "r2", 1e-3, 1.5),
            W.two_level_column(np.array([0.1, 2.0]), 2, 1, 1, "crd", 0.5, 1.0)]


def test_batch_offsets_are_the_cumulative_column_sizes():
    """The batch vector is the columns back to back (each in the ordering of
    Sec. 3.1): offsets start at 0, step by n_z * n_dir * n_nu and end at the
    total length."""
    cols = _ragged_columns()
    off = O.batch_offsets(cols)
    sizes = [c.nz * c.n_dir * c.n_nu for c in cols]
    assert off.tolist() == [0, sizes[0], sizes[0] + sizes[1], sum(sizes)]


def test_batch_apply_is_the_block_diagonal_operator():
    """A batch of independent columns is one block-diagonal system: the
    batched apply equals the block-diagonal matrix of the columns' assembled
    A_N (eq. RT_sys_algebraic) times a random vector, and permuting the
    columns permutes the output blocks the same way."""
    cols = _ragged_columns()
    blocks = [O.assemble_A(c) for c in cols]
    n = sum(b.shape[0] for b in blocks)
    big = np.zeros((n, n))
    o = 0
    for b in blocks:
        big[o:o + b.shape[0], o:o + b.shape[0]] = b
        o += b.shape[0]
    x = np.random.default_rng(3).standard_normal(n)
    y = O.apply_A_batch(cols, x)
    assert np.linalg.norm(y - big @ x) <= 1e-13 * np.linalg.norm(big @ x)
    off = O.batch_offsets(cols)
    perm = [2, 0, 1]
    xp = np.concatenate([x[off[c]:off[c + 1]] for c in perm])
    yp = O.apply_A_batch([cols[c] for c in perm], xp)
    assert np.array_equal(yp, np.concatenate([y[off[c]:off[c + 1]] for c in perm]))


def test_batch_rhs_solves_with_the_column_solutions():
    """b of the batch (Lambda t + I_in per column) solved as one block-diagonal
    system gives each column's own dense solution."""
    cols = _ragged_columns()
    b = O.rhs_batch(cols)
    off = O.batch_offsets(cols)
    assert b.shape == (off[-1],)
    for c, p in enumerate(cols):
        xc = np.linalg.solve(O.assemble_A(p), b[off[c]:off[c + 1]])
        assert np.linalg.norm(xc - O.solve_dense(p)) <= 1e-13 * np.linalg.norm(xc)


# ------------------------------------------------- low-rank Sigma (Sec. 4)
def _lowrank_column():
    return W.two_level_column(np.logspace(-3, 3, 11), 4, 2, 24, "r2", 1e-3, 1.0)


def test_truncated_frequency_kernel_at_zero_tolerance_is_the_kernel():
    p = _lowrank_column()
    Rr, r = O.truncated_frequency_kernel(p, 0.0)
    assert r == p.n_nu
    assert np.abs(Rr - p.R).max() <= 1e-13 * np.abs(p.R).max()
    # Gamma = (1 - eps)/phi amplifies the reconstruction's rounding in the
    # line wings (phi ~ 1e-7 there), hence the looser bar on Sigma itself
    x = W.random_vectors(p.n, 1, 5)[0]
    assert np.linalg.norm(O.sigma_op_lowrank(p, x, 0.0) - O.sigma_op(p, x)) <= 1e-10 * np.linalg.norm(O.sigma_op(p, x))


def test_truncation_error_is_the_largest_dropped_eigenvalue():
    """In the norm weighted by W^(1/2), the error of the truncated R W is the
    largest dropped |eigenvalue| of W^(1/2) R W^(1/2) (Eckart-Young for a
    symmetric matrix), and the rank falls monotonically with the tolerance."""
    p = _lowrank_column()
    sw = np.sqrt(p.w_nu)
    lam = np.linalg.eigvalsh(sw[:, None] * p.R * sw[None, :])
    ranks = []
    for tol in (1e-6, 1e-3, 1e-1):
        Rr, r = O.truncated_frequency_kernel(p, tol)
        ranks.append(r)
        E = sw[:, None] * (p.R - Rr) * sw[None, :]      # W^(1/2) (R - R_r) W^(1/2)
        dropped = np.abs(lam)[np.abs(lam) < tol * np.abs(lam).max()]
        assert r == p.n_nu - dropped.size
        assert abs(np.linalg.norm(E, 2) - (dropped.max() if dropped.size else 0.0)) <= 1e-12 * np.abs(lam).max()
    assert ranks[0] >= ranks[1] >= ranks[2] and ranks[2] < p.n_nu


def test_crd_kernel_is_rank_one():
    """Complete redistribution R = phi phi^T has rank 1: any tolerance below 1
    keeps one eigenvalue and the Sigma is exact."""
    p = W.two_level_column(np.logspace(-2, 2, 6), 4, 2, 9, "crd", 1e-2, 1.0)
    Rr, r = O.truncated_frequency_kernel(p, 1e-3)
    assert r == 1
    x = W.random_vectors(p.n, 1, 6)[0]
    ref = O.sigma_op(p, x)
    # exact up to the reconstruction's rounding, amplified by Gamma = (1 - eps)/phi
    assert np.linalg.norm(O.sigma_op_lowrank(p, x, 1e-3) - ref) <= 1e-10 * np.linalg.norm(ref)
