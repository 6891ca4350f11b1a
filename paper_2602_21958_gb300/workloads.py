"""Seeded synthetic inputs for the discrete-ordinates radiative-transfer operator.

This module only *builds inputs*: grids, quadratures, absorption profiles,
redistribution kernels, opacity fields and right-hand sides.  It holds none of
the operator's arithmetic (no formal solution, no scattering contraction, no
Krylov step); both the CUDA path and the CPU oracle consume what it returns.

Problem model (Sec. 2-3 of the paper, eqs. RT, emissivity, S, Sigma):

* unknown ``I(p, Omega, nu)`` stored lexicographically, point-major, then
  direction, then frequency fastest (the space-based ordering of Sec. 3.1);
* opacity ``chi(p, nu)``: optical depth increment between two points along a
  direction is the trapezoid ``0.5*(chi_u + chi_c) * |dz| / |Omega_z|``;
* scattering ``S(p,Omega,nu) = gamma(p,nu) * sum_{Omega',nu'} P(Omega,Omega')
  w_Omega' R(nu,nu') w_nu' I(p,Omega',nu') + t(p,nu)`` (separable kernel
  ``Phi = P (x) R``), or with a dense kernel matrix ``Psi`` over rays;
* direction weights are normalised to sum 1 (the 1/N_r factor of the paper's
  W_r is folded into the quadrature weights).

Geometry.  A 1D column has ``nz`` points on a depth coordinate ``z`` that
increases from the surface (index 0) to the deep boundary; ``chi`` is per unit
of ``z``.  A 3D box has ``nz`` planes of ``ny*nx`` cells, plane 0 at the top;
point index ``p = (k*ny + j)*nx + i``.  ``Omega_z = mu > 0`` points up (towards
index 0), as the emerging radiation of Sec. 3.

Seeds: numpy PCG64, default ``20262195 + config_id``.
"""
from __future__ import annotations

import dataclasses
import functools
import math
from typing import Optional

import numpy as np

SEED_BASE = 20262195

FS_SCL = "scl"  # linear short-characteristics exponential integrator
FS_IE = "ie"    # implicit Euler (eqs. ie_1, ie_2)
FS_QSC = "qsc"  # quadratic short-characteristics exponential integrator
FS_LC = "lc"    # long characteristics (3D boxes): linear steps along each point's own ray


@dataclasses.dataclass
class Problem:
    """One radiative-transfer problem (a 1D column or a 3D box)."""

    dims: int
    nx: int
    ny: int
    nz: int
    z: np.ndarray          # 1D: depth coordinate [nz]; 3D: spacings (dx, dy, dz)
    dirs: np.ndarray       # [n_dir, 3] unit vectors, column 2 is mu
    w_dir: np.ndarray      # [n_dir], sums to 1
    w_nu: np.ndarray       # [n_nu]
    chi: np.ndarray        # [n_pts, n_nu] opacity
    gamma: np.ndarray      # [n_pts, n_nu] scattering coefficient
    P: Optional[np.ndarray] = None    # [n_dir, n_dir] angular kernel
    R: Optional[np.ndarray] = None    # [n_nu, n_nu] frequency kernel
    Psi: Optional[np.ndarray] = None  # [n_r, n_r] dense ray kernel
    t_src: Optional[np.ndarray] = None  # [n_pts, n_nu] thermal term eps_t/chi
    I_top: Optional[np.ndarray] = None  # [n_nu] inflow through the top (mu < 0)
    I_bot: Optional[np.ndarray] = None  # [n_nu] inflow through the bottom (mu > 0)
    formal_solver: str = FS_SCL
    name: str = ""

    @property
    def n_dir(self) -> int:
        return int(self.dirs.shape[0])

    @property
    def n_nu(self) -> int:
        return int(self.w_nu.shape[0])

    @property
    def n_r(self) -> int:
        return self.n_dir * self.n_nu

    @property
    def n_pts(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n(self) -> int:
        return self.n_pts * self.n_r

    @property
    def mu(self) -> np.ndarray:
        return self.dirs[:, 2]

    @property
    def kernel_kind(self) -> str:
        return "dense" if self.Psi is not None else "separable"

    def with_dense_kernel(self) -> "Problem":
        """Same operator with the separable kernel P (x) R written out as Psi."""
        assert self.P is not None and self.R is not None
        psi = np.kron(self.P, self.R)
        return dataclasses.replace(self, Psi=psi, P=None, R=None)


# ---------------------------------------------------------------- quadratures
def gauss_legendre_directions(n_mu: int, n_azimuth: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """``n_mu`` inclinations (Gauss-Legendre, ``n_mu/2`` on each of [-1,0) and
    (0,1], Sec. 5) times ``n_azimuth`` equispaced azimuths.

    Directions are ordered by ascending mu (mu < 0 first), azimuth fastest.
    Weights sum to 1.
    """
    if n_mu % 2:
        raise ValueError("n_mu must be even")
    x, w = np.polynomial.legendre.leggauss(n_mu // 2)
    mu_pos = 0.5 * (x + 1.0)
    w_pos = 0.5 * w
    order = np.argsort(mu_pos)
    mu_pos, w_pos = mu_pos[order], w_pos[order]
    mu = np.concatenate([-mu_pos[::-1], mu_pos])
    wm = np.concatenate([w_pos[::-1], w_pos]) / 2.0
    phis = 2.0 * np.pi * np.arange(n_azimuth) / n_azimuth
    dirs, wts = [], []
    for m, wk in zip(mu, wm):
        s = math.sqrt(max(0.0, 1.0 - m * m))
        for ph in phis:
            dirs.append((s * math.cos(ph), s * math.sin(ph), m))
            wts.append(wk / n_azimuth)
    return np.asarray(dirs), np.asarray(wts)


# First cosines of the level-symmetric LQ_n sets (Carlson's tables).
_LS_MU1 = {4: 0.3500212, 6: 0.1838670, 8: 0.1422555}


def level_symmetric(order: int) -> tuple[np.ndarray, np.ndarray]:
    """Level-symmetric S_N set: ``order*(order+2)`` directions, weights sum to 1.

    Cosines from mu_i^2 = mu_1^2 + (i-1) * 2(1 - 3 mu_1^2)/(N-2); one weight per
    permutation class, fixed by the even moment conditions sum w = 1 and
    sum w mu_x^(2m) = 1/(2m+1), m = 2..(number of classes).
    """
    if order not in _LS_MU1:
        raise ValueError("supported orders: 4, 6, 8")
    mu1 = _LS_MU1[order]
    nlev = order // 2
    d = 2.0 * (1.0 - 3.0 * mu1 * mu1) / (order - 2)
    mus = np.sqrt(mu1 * mu1 + d * np.arange(nlev))
    pts, cls = [], []
    for i in range(nlev):
        for j in range(nlev):
            k = (nlev - 1) - i - j  # i + j + k = nlev - 1 (0-based level indices)
            if k < 0:
                continue
            pts.append((mus[i], mus[j], mus[k]))
            cls.append(tuple(sorted((i, j, k))))
    classes = sorted(set(cls))
    ncls = len(classes)
    a = np.zeros((ncls, ncls))
    rhs = np.zeros(ncls)
    for c_i, c in enumerate(classes):
        members = [p for p, cc in zip(pts, cls) if cc == c]
        a[0, c_i] = 8.0 * len(members)
        for row in range(1, ncls):
            pw = 2 * (row + 1)
            a[row, c_i] = 8.0 * sum(p[0] ** pw for p in members)
    rhs[0] = 1.0
    for row in range(1, ncls):
        rhs[row] = 1.0 / (2 * (row + 1) + 1)
    wc = np.linalg.solve(a, rhs)
    dirs, wts = [], []
    for sz in (-1.0, 1.0):  # mu < 0 first
        for sy in (-1.0, 1.0):
            for sx in (-1.0, 1.0):
                for p, c in zip(pts, cls):
                    dirs.append((sx * p[0], sy * p[1], sz * p[2]))
                    wts.append(wc[classes.index(c)])
    dirs = np.asarray(dirs)
    wts = np.asarray(wts)
    order_idx = np.lexsort((dirs[:, 1], dirs[:, 0], dirs[:, 2]))
    return dirs[order_idx], wts[order_idx]


def trapezoid_weights(x: np.ndarray) -> np.ndarray:
    """Trapezoid rule weights on a (possibly non-uniform) increasing grid."""
    w = np.zeros_like(x, dtype=float)
    if len(x) == 1:
        w[0] = 1.0
        return w
    dx = np.diff(x)
    w[:-1] += 0.5 * dx
    w[1:] += 0.5 * dx
    return w


# ------------------------------------------------------------------ profiles
def voigt(x: np.ndarray, a: float) -> np.ndarray:
    """Normalised Voigt profile H(a,x)/sqrt(pi), H = Re w(x + i a) (Faddeeva)."""
    from scipy.special import wofz

    return wofz(np.asarray(x, dtype=float) + 1j * a).real / math.sqrt(math.pi)


def lorentz(x: np.ndarray) -> np.ndarray:
    """phi(nu) = 1 / (pi (nu^2 + 1)) (Sec. 5.2)."""
    x = np.asarray(x, dtype=float)
    return 1.0 / (math.pi * (x * x + 1.0))


# ------------------------------------------------------- redistribution kernels
_GL_NODES, _GL_WTS = np.polynomial.legendre.leggauss(24)


def _panel_quadrature(func, brk: np.ndarray) -> np.ndarray:
    """Composite 24-point Gauss-Legendre over sorted breakpoints ``brk`` [m, nb]."""
    lo, hi = brk[:, :-1], brk[:, 1:]
    half = 0.5 * (hi - lo)
    mid = 0.5 * (hi + lo)
    u = mid[..., None] + half[..., None] * _GL_NODES  # [m, panels, nodes]
    return np.sum(func(u) * (half[..., None] * _GL_WTS), axis=(1, 2))


def _graded(center: np.ndarray, a: float) -> list[np.ndarray]:
    out = [center]
    for s in (1.0, 4.0, 16.0, 64.0, 256.0, 1024.0):
        out += [center - s * a, center + s * a]
    return out


def r2a_pairs(xa: np.ndarray, xb: np.ndarray, a: float) -> np.ndarray:
    """Angle-averaged R_II-A (Hummer 1962) at the frequency pairs (xa_k, xb_k).

    R(x,x') = pi^(-3/2) int_{(xh-xl)/2}^inf exp(-u^2)
              [atan((xl+u)/a) - atan((xh-u)/a)] du,
    xh = max(x, x'), xl = min(x, x') (signed: coherent in the wings).
    Normalised: int R dx' = phi(x); a -> 0 gives erfc(max(|x|,|x'|))/2.
    """
    xa, xb = np.asarray(xa, dtype=float), np.asarray(xb, dtype=float)
    xh = np.maximum(xa, xb)
    xl = np.minimum(xa, xb)
    u0 = 0.5 * (xh - xl)
    top = np.maximum(u0, np.maximum(np.abs(xh), np.abs(xl))) + 6.5
    pts = _graded(np.abs(xh), a) + _graded(np.abs(xl), a)
    pts += [u0 + s * a for s in (1.0, 4.0, 16.0, 64.0, 256.0)]
    pts += [np.abs(xh) + 1.0, np.abs(xl) + 1.0, 0.5 * (u0 + np.abs(xh))]
    brk = np.stack([u0, top] + pts, axis=1)
    brk = np.clip(brk, u0[:, None], top[:, None])
    brk.sort(axis=1)

    def f(u):
        return np.exp(-u * u) * (np.arctan((xl[:, None, None] + u) / a)
                                 - np.arctan((xh[:, None, None] - u) / a))

    return _panel_quadrature(f, brk) / math.pi ** 1.5


def r3a_pairs(xa: np.ndarray, xb: np.ndarray, a: float) -> np.ndarray:
    """Angle-averaged R_III-A (Hummer 1962) at the frequency pairs (xa_k, xb_k):

    R(x,x') = pi^(-5/2) int_0^inf exp(-u^2) [atan((x+u)/a) - atan((x-u)/a)]
              [atan((x'+u)/a) - atan((x'-u)/a)] du.   int R dx' = phi(x).
    """
    xa, xb = np.asarray(xa, dtype=float), np.asarray(xb, dtype=float)
    top = np.maximum(np.abs(xa), np.abs(xb)) + 6.5
    zero = np.zeros_like(xa)
    pts = _graded(np.abs(xa), a) + _graded(np.abs(xb), a)
    pts += [zero + s * a for s in (1.0, 4.0, 16.0, 64.0, 256.0)]
    pts += [np.abs(xa) + 1.0, np.abs(xb) + 1.0]
    brk = np.stack([zero, top] + pts, axis=1)
    brk = np.clip(brk, 0.0, top[:, None])
    brk.sort(axis=1)

    def f(u):
        ga = np.arctan((xa[:, None, None] + u) / a) - np.arctan((xa[:, None, None] - u) / a)
        gb = np.arctan((xb[:, None, None] + u) / a) - np.arctan((xb[:, None, None] - u) / a)
        return np.exp(-u * u) * ga * gb

    return _panel_quadrature(f, brk) / math.pi ** 2.5


def _kernel_matrix(fn, x: np.ndarray, a: float) -> np.ndarray:
    x = np.asarray(x, dtype=float)
    n = len(x)
    return fn(np.repeat(x, n), np.tile(x, n), a).reshape(n, n)


def redistribution_r2a(x: np.ndarray, a: float) -> np.ndarray:
    """R_II-A matrix on the reduced-frequency grid ``x`` (see :func:`r2a_pairs`)."""
    return _kernel_matrix(r2a_pairs, x, a)


def redistribution_r3a(x: np.ndarray, a: float) -> np.ndarray:
    """R_III-A matrix on the reduced-frequency grid ``x`` (see :func:`r3a_pairs`)."""
    return _kernel_matrix(r3a_pairs, x, a)


def conserve_symmetric(R: np.ndarray, w: np.ndarray, phi: np.ndarray,
                       iters: int = 2000, tol: float = 1e-15) -> np.ndarray:
    """Symmetric rescaling D R D so that sum_k w_k R_jk = phi_j exactly.

    Keeps R symmetric (Sec. 3.3: Psi is symmetric) while making the discrete
    scattering conservative; fixed point d <- sqrt(d * phi / (R (w d))).
    """
    d = np.ones(len(phi))
    for _ in range(iters):
        m = R @ (w * d)
        d_new = np.sqrt(d * phi / m)
        if np.max(np.abs(d_new / d - 1.0)) < tol:
            d = d_new
            break
        d = d_new
    return d[:, None] * R * d[None, :]


# ------------------------------------------------------------- angular kernels
def legendre_kernel(mu: np.ndarray, coeffs) -> np.ndarray:
    """Phi(mu,mu') = sum_l d_l P_l(mu) P_l(mu') (Sec. 5.1)."""
    from numpy.polynomial import legendre as L

    mu = np.asarray(mu, dtype=float)
    out = np.zeros((len(mu), len(mu)))
    for ell, d in enumerate(coeffs):
        c = np.zeros(ell + 1)
        c[ell] = 1.0
        p = L.legval(mu, c)
        out += d * np.outer(p, p)
    return out


# Legendre coefficients of the monochromatic test kernel, L = 7 (Sec. 5.1).
MONO_LEGENDRE = (1.0, 1.98398, 1.50823, 0.70075, 0.23489, 0.05133, 0.00760, 0.00048)


def dipole_azimuth_averaged(mu: np.ndarray) -> np.ndarray:
    """Azimuth average of 3/4 (1 + cos^2 Theta): 1 + P2(mu) P2(mu') / 2."""
    p2 = 0.5 * (3.0 * mu * mu - 1.0)
    return 1.0 + 0.5 * np.outer(p2, p2)


def dipole_3d(dirs: np.ndarray) -> np.ndarray:
    """Dipole (Rayleigh) phase 3/4 (1 + (Omega . Omega')^2)."""
    c = dirs @ dirs.T
    return 0.75 * (1.0 + c * c)


# ------------------------------------------------------------- random fields
def lognormal_opacity(shape, corr: float, rng: np.random.Generator,
                      kappa0: float = 1.0) -> np.ndarray:
    """kappa = kappa0 * exp(g - 1/2), g a unit-variance Gaussian field: white
    N(0,1) noise smoothed by a periodic separable Gaussian (std ``corr`` cells),
    then shifted/scaled to zero mean and unit standard deviation."""
    g = rng.standard_normal(shape)
    for ax, n in enumerate(shape):
        k = np.fft.fftfreq(n)
        filt = np.exp(-0.5 * (2.0 * np.pi * k * corr) ** 2)
        g = np.fft.ifft(np.fft.fft(g, axis=ax) * filt.reshape(
            [-1 if i == ax else 1 for i in range(len(shape))]), axis=ax).real
    g = (g - g.mean()) / g.std()
    return kappa0 * np.exp(g - 0.5)


# --------------------------------------------------------------- frequency data
@functools.lru_cache(maxsize=256)
def _line_data(n_nu: int, span: float, a: float, kernel: str):
    x = np.linspace(-span, span, n_nu)
    w = trapezoid_weights(x)
    phi = voigt(x, a)
    phi = phi / np.sum(w * phi)
    if kernel == "crd":
        R = np.outer(phi, phi)
    elif kernel == "r2":
        R = conserve_symmetric(redistribution_r2a(x, a), w, phi)
    elif kernel == "r23":
        R = 0.7 * redistribution_r2a(x, a) + 0.3 * redistribution_r3a(x, a)
        R = conserve_symmetric(0.5 * (R + R.T), w, phi)
    else:
        raise ValueError(kernel)
    return x, w, phi, R


def line_data(n_nu: int, kernel: str, span: float = 5.0, a: float = 1e-3):
    """Reduced-frequency grid on [-span, span], trapezoid weights, Voigt profile
    renormalised to sum w phi = 1, and the conservative frequency kernel."""
    x, w, phi, R = _line_data(int(n_nu), float(span), float(a), kernel)
    return x.copy(), w.copy(), phi.copy(), R.copy()


# ------------------------------------------------------------ two-level columns
def two_level_column(t: np.ndarray, n_mu: int, n_azimuth: int, n_nu: int,
                     kernel: str, eps, B, name: str = "",
                     formal_solver: str = FS_SCL) -> Problem:
    """1D plane-parallel two-level-atom column on the optical-depth grid ``t``.

    chi(t, nu) = phi(nu); gamma = (1 - eps)/phi; t_src = eps B; P the
    azimuth-averaged dipole (or isotropic when n_azimuth == 1 and kernel is
    'crd'); inflow 0 at the surface and B at the deep boundary.
    """
    t = np.asarray(t, dtype=float)
    nz = len(t)
    dirs, wd = gauss_legendre_directions(n_mu, n_azimuth)
    x, wn, phi, R = line_data(n_nu, kernel)
    eps = np.broadcast_to(np.asarray(eps, dtype=float), (nz,)).copy()
    Bv = np.broadcast_to(np.asarray(B, dtype=float), (nz,)).copy()
    if kernel == "crd" and n_azimuth == 1:
        P = np.ones((len(wd), len(wd)))
    else:
        P = dipole_azimuth_averaged(dirs[:, 2])
    chi = np.tile(phi, (nz, 1))
    gamma = (1.0 - eps)[:, None] / phi[None, :]
    t_src = np.tile((eps * Bv)[:, None], (1, n_nu))
    return Problem(dims=1, nx=1, ny=1, nz=nz, z=t, dirs=dirs, w_dir=wd, w_nu=wn,
                   chi=chi, gamma=gamma, P=P, R=R, t_src=t_src,
                   I_top=np.zeros(n_nu), I_bot=np.full(n_nu, Bv[-1]),
                   formal_solver=formal_solver, name=name)


def config_c1() -> Problem:
    """Slab, CRD, isotropic: 64 log-spaced t in [1e-4, 1e4], 4+4 GL, 21 nu."""
    t = np.logspace(-4, 4, 64)
    return two_level_column(t, 8, 1, 21, "crd", 1e-4, 1.0, name="C1")


def _b_linear_log(t):
    lt = np.log(t)
    return 1.0 + (lt - lt[0]) / (lt[-1] - lt[0])


def config_c2(seed: Optional[int] = None) -> Problem:
    """Slab, dipole x R_II-A: 128 log t in [1e-6, 1e6], 16 dirs, 64 nu,
    eps i.i.d. log-uniform in [1e-6, 1e-2] per depth point, B linear in log t."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 2 if seed is None else seed))
    t = np.logspace(-6, 6, 128)
    eps = 10.0 ** rng.uniform(-6, -2, size=len(t))
    return two_level_column(t, 8, 2, 64, "r2", eps, _b_linear_log(t), name="C2")


def _c5_params(seed: Optional[int], n_col: int, nz_range, nnu_range):
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 5 if seed is None else seed))
    nzs = rng.integers(nz_range[0], nz_range[1] + 1, size=n_col)
    nnus = rng.integers(nnu_range[0], nnu_range[1] + 1, size=n_col)
    epss = 10.0 ** rng.uniform(-6, -2, size=n_col)
    return nzs, nnus, epss


def config_c5_column(ci: int, seed: Optional[int] = None, n_col: int = 256,
                     nz_range=(64, 512), nnu_range=(32, 128)) -> Problem:
    """Column ``ci`` of :func:`config_c5` (same seed stream), built alone."""
    nzs, nnus, epss = _c5_params(seed, n_col, nz_range, nnu_range)
    t = np.logspace(-4, 4, int(nzs[ci]))
    return two_level_column(t, 8, 2, int(nnus[ci]), "r2", float(epss[ci]),
                            _b_linear_log(t), name=f"C5[{ci}]")


def config_c5(seed: Optional[int] = None, n_col: int = 256,
              nz_range=(64, 512), nnu_range=(32, 128)) -> list[Problem]:
    """Ragged batch of slabs: N_z ~ U{64..512} log-spaced points over t in
    [1e-4, 1e4] (the slab range of the CRD test column), N_nu ~ U{32..128},
    16 dirs, dipole x R_II-A, one log-uniform eps in [1e-6, 1e-2] per column,
    B linear in log t."""
    return [config_c5_column(c, seed, n_col, nz_range, nnu_range) for c in range(n_col)]


def c5_random_rhs(ci: int, rhs: int, n: int, seed: Optional[int] = None) -> np.ndarray:
    """Seeded N(0,1) right-hand side of instance (column ci, rhs >= 1) of the
    ragged batch, drawn per instance so any instance can be rebuilt alone."""
    base = SEED_BASE + 55 if seed is None else seed
    rng = np.random.Generator(np.random.PCG64([base, ci, rhs]))
    return rng.standard_normal(n)


def box_3d(n: int, order: int, n_nu: int, kernel: str, eps: float, seed: int,
           corr: float = 4.0, name: str = "", nz: Optional[int] = None) -> Problem:
    """Periodic-in-x,y box of n x n x nz unit cells (nz = n by default),
    level-symmetric S_order directions, dipole phase, lognormal opacity
    kappa(p) phi(nu), open top (I=0) and bottom (I=B=1), gamma = (1-eps)/phi,
    t = eps B."""
    nz = n if nz is None else nz
    rng = np.random.Generator(np.random.PCG64(seed))
    kappa = lognormal_opacity((nz, n, n), corr, rng).ravel()
    dirs, wd = level_symmetric(order)
    x, wn, phi, R = line_data(n_nu, kernel)
    npts = n * n * nz
    chi = kappa[:, None] * phi[None, :]
    gamma = np.tile((1.0 - eps) / phi, (npts, 1))
    t_src = np.full((npts, n_nu), eps * 1.0)
    return Problem(dims=3, nx=n, ny=n, nz=nz, z=np.array([1.0, 1.0, 1.0]), dirs=dirs,
                   w_dir=wd, w_nu=wn, chi=chi, gamma=gamma, P=dipole_3d(dirs), R=R,
                   t_src=t_src, I_top=np.zeros(n_nu), I_bot=np.ones(n_nu),
                   formal_solver=FS_SCL, name=name)


def config_c3(n: int = 32) -> Problem:
    """3D box, 32^3, S_6 (48 dirs), 32 nu, dipole x CRD, eps = 1e-3."""
    return box_3d(n, 6, 32, "crd", 1e-3, SEED_BASE + 3, name=f"C3[{n}^3]")


def config_c4(n: int = 64) -> Problem:
    """3D box, 64^3, S_8 (80 dirs), 64 nu, dipole x (0.7 R_II-A + 0.3 R_III-A)."""
    return box_3d(n, 8, 64, "r23", 1e-3, SEED_BASE + 4, name=f"C4[{n}^3]")


# ---------------------------------------------------- the paper's 1D test setups
def paper_mono(n_s: int, n_omega: int, formal_solver: str = FS_IE) -> Problem:
    """Monochromatic test of Sec. 5.1: equidistant t on [0,1], GL directions,
    Legendre kernel (L = 7), gamma = (1 - t)/2 with the angular weights
    normalised to sum 1 (the reading that reproduces Table mono), phi = 1."""
    t = np.linspace(0.0, 1.0, n_s)
    dirs, wd = gauss_legendre_directions(n_omega, 1)
    P = legendre_kernel(dirs[:, 2], MONO_LEGENDRE)
    gamma = 0.5 * (1.0 - t)[:, None]
    return Problem(dims=1, nx=1, ny=1, nz=n_s, z=t, dirs=dirs, w_dir=wd,
                   w_nu=np.ones(1), chi=np.ones((n_s, 1)), gamma=gamma, P=P,
                   R=np.ones((1, 1)), t_src=None, I_top=np.zeros(1), I_bot=np.ones(1),
                   formal_solver=formal_solver, name=f"mono[{n_s},{n_omega}]")


def paper_iso(n_s: int, n_nu: int, kind: str, n_mu: int = 12,
              formal_solver: str = FS_IE, span: float = 10.0) -> Problem:
    """Isotropic tests of Sec. 5.2: equidistant t on [0,1], Lorentz profile on
    [-10, 10] (trapezoid), gamma*phi = (1 - t)/2 against the angular integral
    over [-1, 1] (GL weights summing to 2; stored weights sum to 1, so the
    stored gamma*phi is 1 - t: the reading that reproduces the GMRES counts).

    kind 'coherent': Phi = phi(nu') delta(nu - nu')  ->  R = diag(phi / w_nu);
    kind 'crd':      Phi = phi(nu) phi(nu')          ->  R = phi phi^T.
    """
    t = np.linspace(0.0, 1.0, n_s)
    dirs, wd = gauss_legendre_directions(n_mu, 1)
    x = np.linspace(-span, span, n_nu)
    wn = trapezoid_weights(x)
    phi = lorentz(x)
    if kind == "coherent":
        R = np.diag(phi / wn)
    elif kind == "crd":
        R = np.outer(phi, phi)
    else:
        raise ValueError(kind)
    P = np.ones((n_mu, n_mu))
    gamma = (1.0 - t)[:, None] / phi[None, :]
    return Problem(dims=1, nx=1, ny=1, nz=n_s, z=t, dirs=dirs, w_dir=wd, w_nu=wn,
                   chi=np.tile(phi, (n_s, 1)), gamma=gamma, P=P, R=R, t_src=None,
                   I_top=np.zeros(n_nu), I_bot=np.ones(n_nu),
                   formal_solver=formal_solver, name=f"iso-{kind}[{n_s},{n_nu}]")


# ----------------------------------------------------------------- vectors
def random_vectors(n: int, count: int, seed: int, kind: str = "normal") -> np.ndarray:
    """Seeded test vectors [count, n]: 'normal' N(0,1) or 'uniform' U[0,1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "normal":
        return rng.standard_normal((count, n))
    return rng.uniform(0.0, 1.0, size=(count, n))
