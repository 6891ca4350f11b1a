"""Plain, slow FP64 restatement of the S_N radiative-transfer operator and its
solve (test infrastructure only; see the package docstring).

Notation follows the paper: Lambda_N is the formal solver (Sec. 3.2, eqs.
ie_1, ie_2, lambda_block), Sigma_N = Gamma_N Psi_N W_N the scattering
operator (Sec. 3.3, eqs. S, Sigma), A_N = Id - Lambda_N Sigma_N and
b = Lambda_N t + I_in (eq. RT_sys_algebraic).  Vectors use the space-based
lexicographic ordering (point, direction, frequency fastest) of Sec. 3.1.

Readings where the paper is silent or garbled:
* the formal solver is the linear short-characteristics exponential
  integrator (SC-L) unless the problem asks for implicit Euler (IE); the paper
  allows any formal solver (Sec. 3.2, final remark);
* the inflow vector I_in is the boundary intensity propagated by Lambda with
  S = 0 (the matrix forms after eq. ie_mono4), not a vector that is non-zero
  only in its first and last blocks;
* optical-depth increments are trapezoids of chi along the ray;
* in 3D, rays are short characteristics between consecutive z-planes with
  bilinear interpolation (periodic in x and y) of I, S and chi at the upwind
  point (the interpolation operators T_RC, T_CR of Sec. 3.4, rows summing to 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from paper_2602_21958_gb300.workloads import FS_IE, FS_LC, FS_QSC, FS_SCL, Problem

SERIES_CUT = 0.1


# ------------------------------------------------------------ formal solvers
def w1_over_dtau(d: np.ndarray) -> np.ndarray:
    """w1/dtau with w1 = dtau - (1 - e^-dtau) = int_0^dtau s e^-(dtau-s) ds / ...
    (the linear-source weight of the SC-L step; Sec. 3.2 admits any formal solver).

    For dtau < 0.1 the alternating series sum_{k>=1} (-1)^(k+1) dtau^k/(k+1)!
    (16 terms) replaces the cancelling closed form.
    """
    d = np.asarray(d, dtype=float)
    out = np.empty_like(d)
    small = d < SERIES_CUT
    ds = d[small]
    acc = np.zeros_like(ds)
    term = np.ones_like(ds)
    for k in range(1, 17):
        term = term * ds / (k + 1)        # dtau^k / (k+1)!
        acc += term if k % 2 == 1 else -term
    out[small] = acc
    dl = d[~small]
    out[~small] = (dl + np.expm1(-dl)) / dl
    return out


def step_coefficients(dtau: np.ndarray, formal_solver: str):
    """Coefficients (e, alpha, beta) of one step I_c = e I_u + alpha S_u + beta S_c.

    IE (eqs. ie_1, ie_2): I_c = (I_u + dtau S_c)/(1 + dtau).
    SC-L: S linear between the upwind and the current point, integrated exactly
    against e^-(dtau - s): e = e^-dtau, w0 = 1 - e (= -expm1(-dtau)),
    beta = w1/dtau, alpha = w0 - beta.
    """
    dtau = np.asarray(dtau, dtype=float)
    if formal_solver == FS_IE:
        e = 1.0 / (1.0 + dtau)
        return e, np.zeros_like(dtau), dtau * e
    if formal_solver != FS_SCL:
        raise ValueError(formal_solver)
    e = np.exp(-dtau)
    w0 = -np.expm1(-dtau)
    beta = w1_over_dtau(dtau)
    return e, w0 - beta, beta


def qsc_moments(d: np.ndarray):
    """Moments of the quadratic step (the quadratic integrator of Sec. 5.3, restated):
    W1 = int_0^d s e^-(d-s) ds = d - (1 - e^-d) and W2 = int_0^d s^2 e^-(d-s) ds
    = d^2 - 2 W1, returned as W1/d^2 and W2/d^3.  Below d = 0.1 the cancelling
    closed forms are replaced by their series, W1/d^2 = sum_{k>=0} (-1)^k
    d^k/(k+2)! and W2/d^3 = 2 sum_{k>=0} (-1)^k d^k/(k+3)! (18 terms)."""
    d = np.asarray(d, dtype=float)
    a = np.empty_like(d)
    b = np.empty_like(d)
    small = d < SERIES_CUT
    ds = d[small]
    sa = np.zeros_like(ds)
    sb = np.zeros_like(ds)
    for k in range(18):
        sa += (-1) ** k * ds ** k / math.factorial(k + 2)
        sb += (-1) ** k * ds ** k / math.factorial(k + 3)
    a[small] = sa
    b[small] = 2.0 * sb
    dl = d[~small]
    w1 = dl + np.expm1(-dl)
    a[~small] = w1 / dl ** 2
    b[~small] = (dl ** 2 - 2.0 * w1) / dl ** 3
    return a, b


def qsc_coefficients(du: np.ndarray, dd: np.ndarray):
    """Quadratic short-characteristics step (Sec. 3.2 allows any formal solver;
    the paper's 3D runs use a quadratic exponential integrator, Sec. 5.3):
    S is the parabola through the upwind (u), current (c) and downwind (d)
    points, at path depths s = 0, du, du + dd from u, integrated exactly
    against e^-(du - s):  I_c = e I_u + psi_u S_u + psi_c S_c + psi_d S_d with
        psi_c = (W1 (du + dd) - W2) / (du dd)
        psi_d = (W2 - du W1) / (dd (du + dd))
        psi_u = w0 - psi_c - psi_d          (the weights integrate 1 to w0)
    (Lagrange weights integrated with the moments W0 = w0, W1, W2)."""
    du = np.asarray(du, dtype=float)
    dd = np.asarray(dd, dtype=float)
    a, b = qsc_moments(du)          # W1 = du^2 a, W2 = du^3 b
    e = np.exp(-du)
    w0 = -np.expm1(-du)
    pc = du * ((du + dd) * a - du * b) / dd
    pd = du ** 3 * (b - a) / (dd * (du + dd))
    pu = w0 - pc - pd
    return e, pu, pc, pd


# ---------------------------------------------------------------- 1D transfer
def dtau_1d(prob: Problem) -> np.ndarray:
    """Delta tau_i(mu, nu) between depth points i and i+1: [nz-1, n_dir, n_nu].

    In Sec. 5 tau = phi(nu) t / |mu|; with a depth-dependent chi the increment
    is the trapezoid 0.5 (chi_i + chi_{i+1}) (z_{i+1} - z_i) / |mu|.
    """
    dz = np.diff(prob.z)
    cbar = 0.5 * (prob.chi[:-1] + prob.chi[1:])          # [nz-1, n_nu]
    return (cbar * dz[:, None])[:, None, :] / np.abs(prob.mu)[None, :, None]


def lambda_1d(prob: Problem, S: np.ndarray, with_inflow: bool = False) -> np.ndarray:
    """Formal solution I = Lambda S (+ I_in) for a 1D column (eqs. ie_1, ie_2,
    lamda_down, lamda_up).

    mu < 0 rays start at the surface (i = 0) and march down; mu > 0 rays start
    at the deep boundary and march up.  Without inflow the first point of each
    ray is 0 (first row of Lambda_down and last row of Lambda_up are zero).
    """
    nz, nd, nn = prob.nz, prob.n_dir, prob.n_nu
    S = np.asarray(S, dtype=float).reshape(nz, nd, nn)
    if prob.formal_solver == FS_QSC:
        return _lambda_1d_qsc(prob, S, with_inflow)
    e, al, be = step_coefficients(dtau_1d(prob), prob.formal_solver)
    I = np.zeros_like(S)
    down = prob.mu < 0
    up = ~down
    if with_inflow:
        I[0, down, :] = prob.I_top[None, :]
        I[nz - 1, up, :] = prob.I_bot[None, :]
    for i in range(1, nz):                     # mu < 0: upwind i-1, current i
        I[i, down] = (e[i - 1, down] * I[i - 1, down] + al[i - 1, down] * S[i - 1, down]
                      + be[i - 1, down] * S[i, down])
    for i in range(nz - 2, -1, -1):            # mu > 0: upwind i+1, current i
        I[i, up] = (e[i, up] * I[i + 1, up] + al[i, up] * S[i + 1, up]
                    + be[i, up] * S[i, up])
    return I.reshape(-1)


def _lambda_1d_qsc(prob: Problem, S: np.ndarray, with_inflow: bool) -> np.ndarray:
    """Quadratic short characteristics along every ray (Sec. 5.3 integrator,
    recurrence of eqs. ie_1, ie_2 with a downwind term): each step uses the
    upwind, current and downwind points (qsc_coefficients); the last step of a
    ray, which has no downwind point, is the linear SC-L step."""
    nz = prob.nz
    dt = dtau_1d(prob)                               # [nz-1, n_dir, n_nu]
    I = np.zeros_like(S)
    down = prob.mu < 0
    up = ~down
    if with_inflow:
        I[0, down, :] = prob.I_top[None, :]
        I[nz - 1, up, :] = prob.I_bot[None, :]
    for i in range(1, nz):                           # mu < 0: u = i-1, c = i, d = i+1
        du = dt[i - 1, down]
        if i < nz - 1:
            e, pu, pc, pd = qsc_coefficients(du, dt[i, down])
            src = pu * S[i - 1, down] + pc * S[i, down] + pd * S[i + 1, down]
        else:
            e, al, be = step_coefficients(du, FS_SCL)
            src = al * S[i - 1, down] + be * S[i, down]
        I[i, down] = e * I[i - 1, down] + src
    for i in range(nz - 2, -1, -1):                  # mu > 0: u = i+1, c = i, d = i-1
        du = dt[i, up]
        if i > 0:
            e, pu, pc, pd = qsc_coefficients(du, dt[i - 1, up])
            src = pu * S[i + 1, up] + pc * S[i, up] + pd * S[i - 1, up]
        else:
            e, al, be = step_coefficients(du, FS_SCL)
            src = al * S[i + 1, up] + be * S[i, up]
        I[i, up] = e * I[i + 1, up] + src
    return I.reshape(-1)


def lambda_matrix_1d(prob: Problem) -> np.ndarray:
    """Dense Lambda_N (N x N) assembled from the step recurrence, ray by ray,
    in the space-based ordering (Lambda_N = P^T blockdiag(Lambda_[k]) P;
    Sec. 3.2, eq. lambda_block)."""
    nz, nd, nn = prob.nz, prob.n_dir, prob.n_nu
    N = prob.n
    if prob.formal_solver == FS_QSC:  # columns of the matrix-free operator
        return np.stack([lambda_1d(prob, np.eye(1, N, k).ravel()) for k in range(N)], axis=1)
    e, al, be = step_coefficients(dtau_1d(prob), prob.formal_solver)
    L = np.zeros((N, N))
    for d in range(nd):
        for f in range(nn):
            blk = np.zeros((nz, nz))
            if prob.mu[d] < 0:
                for i in range(1, nz):
                    blk[i] = e[i - 1, d, f] * blk[i - 1]
                    blk[i, i - 1] += al[i - 1, d, f]
                    blk[i, i] += be[i - 1, d, f]
            else:
                for i in range(nz - 2, -1, -1):
                    blk[i] = e[i, d, f] * blk[i + 1]
                    blk[i, i + 1] += al[i, d, f]
                    blk[i, i] += be[i, d, f]
            idx = np.arange(nz) * prob.n_r + d * nn + f
            L[np.ix_(idx, idx)] = blk
    return L


def lambda_ie_closed_form(prob: Problem) -> np.ndarray:
    """Dense Lambda_N from the closed-form entries of eqs. ie_mono3 and
    ie_mono4 (implicit Euler): f_{i,j} = dtau_{j-1} / prod_{l=j}^{i}(1+dtau_{l-1})
    for mu < 0 and h_{i,j} = dtau_j / prod_{l=i}^{j}(1+dtau_l) for mu > 0."""
    nz, nd, nn = prob.nz, prob.n_dir, prob.n_nu
    dt = dtau_1d(prob)                       # dt[l] = tau_{l+1} - tau_l (0-based)
    N = prob.n
    L = np.zeros((N, N))
    for d in range(nd):
        for f in range(nn):
            blk = np.zeros((nz, nz))
            D = dt[:, d, f]
            for i in range(nz):
                if prob.mu[d] < 0:
                    for j in range(1, i + 1):         # paper: i, j >= 2 (1-based)
                        blk[i, j] = D[j - 1] / np.prod(1.0 + D[j - 1:i])
                else:
                    for j in range(i, nz - 1):        # paper: j <= N_s - 1
                        blk[i, j] = D[j] / np.prod(1.0 + D[i:j + 1])
            idx = np.arange(nz) * prob.n_r + d * nn + f
            L[np.ix_(idx, idx)] = blk
    return L


# ---------------------------------------------------------------- 3D transfer
def _bilinear_periodic(F: np.ndarray, sx: float, sy: float) -> np.ndarray:
    """Value of the periodic plane field F[..., ny, nx] at (x - sx, y - sy) for
    every cell (x, y), by bilinear interpolation (weights sum to 1): the
    interpolation operators T_RC / T_CR of Sec. 3.4."""
    fx, fy = math.floor(sx), math.floor(sy)
    ax, ay = sx - fx, sy - fy
    # point x - sx = x - fx - ax lies between x - fx - 1 (weight ax) and x - fx
    f00 = np.roll(F, shift=(fy, fx), axis=(-2, -1))          # F[y - fy, x - fx]
    f01 = np.roll(F, shift=(fy, fx + 1), axis=(-2, -1))      # F[y - fy, x - fx - 1]
    f10 = np.roll(F, shift=(fy + 1, fx), axis=(-2, -1))      # F[y - fy - 1, x - fx]
    f11 = np.roll(F, shift=(fy + 1, fx + 1), axis=(-2, -1))
    return ((1 - ay) * ((1 - ax) * f00 + ax * f01) + ay * ((1 - ax) * f10 + ax * f11))


def lambda_3d(prob: Problem, S: np.ndarray, with_inflow: bool = False) -> np.ndarray:
    """Short-characteristics formal solution in a box periodic in x, y (Sec.
    3.4 with T_RC/T_CR realised as bilinear interpolation in the upwind plane).

    For direction Omega with Omega_z > 0 (up) the upwind point of cell (k, y, x)
    is in plane k+1, shifted by -(Omega_x, Omega_y) dz/|Omega_z| (in cell
    units); with Omega_z < 0 it is in plane k-1.  Along the segment
    ds = dz/|Omega_z| the optical depth is 0.5 (chi_u + chi_c) ds and the step
    is the 1D recurrence.  Inflow planes are 0 unless ``with_inflow``.

    Quadratic short characteristics (FS_QSC, the Sec. 5.3 integrator): the
    downwind point continues the ray one segment past the cell, into the next
    plane at the opposite shift +(Omega_x, Omega_y) dz/|Omega_z|; S and chi
    there are interpolated the same way, the downwind optical depth is
    0.5 (chi_c + chi_d) ds, and the step takes qsc_coefficients.  The last
    plane a ray reaches has no downwind point and takes the linear step.
    """
    nx, ny, nz, nd, nn = prob.nx, prob.ny, prob.nz, prob.n_dir, prob.n_nu
    dx, dy, dz = (float(v) for v in prob.z)
    S = np.asarray(S, dtype=float).reshape(nz, ny, nx, nd, nn)
    chi = prob.chi.reshape(nz, ny, nx, nn)
    I = np.zeros_like(S)
    for d in range(nd):
        ox, oy, oz = prob.dirs[d]
        ds = dz / abs(oz)
        sx, sy = ox * ds / dx, oy * ds / dy
        if oz > 0:
            order, first, prev = range(nz - 2, -1, -1), nz - 1, +1
            inflow = prob.I_bot
        else:
            order, first, prev = range(1, nz), 0, -1
            inflow = prob.I_top
        # planes as [n_nu, ny, nx] for the roll-based interpolation
        Iplane = np.zeros((nn, ny, nx))
        if with_inflow:
            Iplane[:] = inflow[:, None, None]
        I[first, :, :, d, :] = np.moveaxis(Iplane, 0, -1)
        for k in order:
            ku = k + prev
            Su = _bilinear_periodic(np.moveaxis(S[ku, :, :, d, :], -1, 0), sx, sy)
            cu = _bilinear_periodic(np.moveaxis(chi[ku], -1, 0), sx, sy)
            Iu = _bilinear_periodic(Iplane, sx, sy)
            Sc = np.moveaxis(S[k, :, :, d, :], -1, 0)
            cc = np.moveaxis(chi[k], -1, 0)
            dtau = 0.5 * (cu + cc) * ds
            kd = k - prev                                  # downwind plane
            if prob.formal_solver == FS_QSC and 0 <= kd < nz:
                Sd = _bilinear_periodic(np.moveaxis(S[kd, :, :, d, :], -1, 0), -sx, -sy)
                cd = _bilinear_periodic(np.moveaxis(chi[kd], -1, 0), -sx, -sy)
                e, pu, pc, pd = qsc_coefficients(dtau, 0.5 * (cc + cd) * ds)
                Iplane = e * Iu + pu * Su + pc * Sc + pd * Sd
            else:
                fs = FS_SCL if prob.formal_solver == FS_QSC else prob.formal_solver
                e, al, be = step_coefficients(dtau, fs)
                Iplane = e * Iu + al * Su + be * Sc
            I[k, :, :, d, :] = np.moveaxis(Iplane, 0, -1)
    return I.reshape(-1)


def lambda_3d_lc(prob: Problem, S: np.ndarray, with_inflow: bool = False) -> np.ndarray:
    """Long characteristics in a box periodic in x, y (the rays of Sec. 3.4
    followed from boundary to point, TRIP's treatment of the 3D transfer named
    in Sec. 5.3): the value at cell (k, y, x) in direction Omega comes from the
    straight ray through that cell traced back to the inflow plane.  That ray
    crosses plane k' (between the inflow plane and k) at the cell position
    shifted back by (k - k') (Omega_x, Omega_y) dz/|Omega_z|; S and chi there
    are interpolated bilinearly (periodic), the intensity never is.  Along the
    ray the linear SC-L step of eqs. ie_1/ie_2's recurrence is taken from
    crossing to crossing, optical depth 0.5 (chi_a + chi_b) ds per segment,
    starting from the inflow (0 unless ``with_inflow``)."""
    nx, ny, nz, nd, nn = prob.nx, prob.ny, prob.nz, prob.n_dir, prob.n_nu
    dx, dy, dz = (float(v) for v in prob.z)
    S = np.asarray(S, dtype=float).reshape(nz, ny, nx, nd, nn)
    chi = prob.chi.reshape(nz, ny, nx, nn)
    I = np.zeros_like(S)
    for d in range(nd):
        ox, oy, oz = prob.dirs[d]
        seg = dz / abs(oz)                          # path length between planes
        sx, sy = ox * seg / dx, oy * seg / dy       # cells per plane
        first, step = (nz - 1, -1) if oz > 0 else (0, 1)
        inflow = prob.I_bot if oz > 0 else prob.I_top
        I0 = np.zeros((nn, ny, nx))
        if with_inflow:
            I0[:] = inflow[:, None, None]
        I[first, :, :, d, :] = np.moveaxis(I0, 0, -1)
        for s in range(1, nz):                      # target plane first + s * step
            Iray = I0.copy()
            Sa = ca = None
            for m in range(s + 1):                  # crossing m: plane first + m * step
                km = first + m * step
                t = s - m                           # segments between the crossing and the target
                Sm = _bilinear_periodic(np.moveaxis(S[km, :, :, d, :], -1, 0), t * sx, t * sy)
                cm = _bilinear_periodic(np.moveaxis(chi[km], -1, 0), t * sx, t * sy)
                if m > 0:
                    e, al, be = step_coefficients(0.5 * (ca + cm) * seg, FS_SCL)
                    Iray = e * Iray + al * Sa + be * Sm
                Sa, ca = Sm, cm
            I[first + s * step, :, :, d, :] = np.moveaxis(Iray, 0, -1)
    return I.reshape(-1)


def lambda_op(prob: Problem, S: np.ndarray, with_inflow: bool = False) -> np.ndarray:
    """Lambda_N S (+ I_in) for a 1D column or a 3D box (Sec. 3.2, Sec. 3.4)."""
    if prob.dims == 1:
        return lambda_1d(prob, S, with_inflow)
    if prob.formal_solver == FS_LC:
        return lambda_3d_lc(prob, S, with_inflow)
    return lambda_3d(prob, S, with_inflow)


# ------------------------------------------------------------------ scattering
def sigma_op(prob: Problem, X: np.ndarray, with_source: bool = False) -> np.ndarray:
    """S = Sigma_N X (+ t): per point p, S_p = Gamma_p Psi W X_p (eq. Sigma).

    Separable kernel Phi = P (x) R: Psi W X_p = (P diag(w_dir)) X_p
    (R diag(w_nu))^T with X_p viewed as [n_dir, n_nu]; dense kernel:
    Psi diag(w_r) X_p with w_r = w_dir (x) w_nu.
    """
    npts, nd, nn = prob.n_pts, prob.n_dir, prob.n_nu
    X = np.asarray(X, dtype=float).reshape(npts, nd, nn)
    if prob.Psi is not None:
        wr = np.kron(prob.w_dir, prob.w_nu)
        Y = (X.reshape(npts, nd * nn) * wr[None, :]) @ prob.Psi.T
        Y = Y.reshape(npts, nd, nn)
    else:
        Pw = prob.P * prob.w_dir[None, :]
        Rw = prob.R * prob.w_nu[None, :]
        Y = np.einsum("ab,pbn,cn->pac", Pw, X, Rw, optimize=True)
    S = prob.gamma[:, None, :] * Y
    if with_source and prob.t_src is not None:
        S = S + prob.t_src[:, None, :]
    return S.reshape(-1)


def truncated_frequency_kernel(prob: Problem, tol: float) -> tuple[np.ndarray, int]:
    """Low-rank frequency kernel for the compressed Sigma (Sec. 4, Remark
    comput: the scattering operator is approximated at rank r_eps with linear
    cost).  The frequency part of Sigma applies R W (W = diag(w_nu)).  It is
    truncated in the W-weighted eigenbasis: M = W^(1/2) R W^(1/2) = U L U^T
    (symmetric R), keeping the eigenvalues with |l| >= tol max |l|, so that
    R_r W = W^(-1/2) U_r L_r U_r^T W^(1/2) is the best rank-r approximation of
    R W in the norm weighted by W^(1/2).  tol = 0 keeps every eigenvalue.
    Returns R_r and r."""
    sw = np.sqrt(prob.w_nu)
    M = sw[:, None] * prob.R * sw[None, :]
    lam, U = np.linalg.eigh(0.5 * (M + M.T))
    keep = np.abs(lam) >= tol * np.abs(lam).max() if tol > 0 else np.ones(lam.size, dtype=bool)
    Ur, lr = U[:, keep], lam[keep]
    Rr = (Ur * lr[None, :]) @ Ur.T / (sw[:, None] * sw[None, :])
    return Rr, int(keep.sum())


def sigma_op_lowrank(prob: Problem, X: np.ndarray, tol: float) -> np.ndarray:
    """Sigma_N X (eq. Sigma) with the frequency kernel replaced by its
    truncation (truncated_frequency_kernel); separable kernels only."""
    if prob.Psi is not None:
        raise ValueError("the low-rank Sigma needs a separable kernel P (x) R")
    Rr, _ = truncated_frequency_kernel(prob, tol)
    from dataclasses import replace
    return sigma_op(replace(prob, R=Rr), X)


def sigma_matrix(prob: Problem) -> np.ndarray:
    """Dense Sigma_N = Gamma_N Psi_N (Id (x) W_r) (eq. Sigma), block diagonal."""
    nd, nn, nr = prob.n_dir, prob.n_nu, prob.n_r
    psi = prob.Psi if prob.Psi is not None else np.kron(prob.P, prob.R)
    wr = np.kron(prob.w_dir, prob.w_nu)
    N = prob.n
    Sg = np.zeros((N, N))
    for p in range(prob.n_pts):
        g = np.tile(prob.gamma[p], nd)
        sl = slice(p * nr, (p + 1) * nr)
        Sg[sl, sl] = g[:, None] * psi * wr[None, :]
    return Sg


# --------------------------------------------------------------- global system
def apply_A(prob: Problem, x: np.ndarray) -> np.ndarray:
    """y = A_N x = x - Lambda_N Sigma_N x (eq. RT_sys_algebraic)."""
    return np.asarray(x, dtype=float) - lambda_op(prob, sigma_op(prob, x))


def rhs(prob: Problem) -> np.ndarray:
    """b = Lambda_N t + I_in (eq. RT_sys_algebraic); I_in is the inflow
    propagated with S = 0."""
    t = np.zeros(prob.n)
    if prob.t_src is not None:
        t = np.broadcast_to(prob.t_src[:, None, :],
                            (prob.n_pts, prob.n_dir, prob.n_nu)).reshape(-1)
    return lambda_op(prob, t) + lambda_op(prob, np.zeros(prob.n), with_inflow=True)


def assemble_A(prob: Problem) -> np.ndarray:
    """Dense A_N = Id - Lambda_N Sigma_N (eq. A_N; 1D only, tiny sizes)."""
    return np.eye(prob.n) - lambda_matrix_1d(prob) @ sigma_matrix(prob)


def solve_dense(prob: Problem, b: np.ndarray | None = None) -> np.ndarray:
    """I = A_N^{-1} b by LU with partial pivoting (LAPACK getrf/getrs): the
    exact solution of eq. RT_sys_algebraic at tiny sizes."""
    A = assemble_A(prob)
    return np.linalg.solve(A, rhs(prob) if b is None else b)


# ---------------------------------------------------------------------- GMRES
@dataclass
class GmresResult:
    x: np.ndarray
    iterations: int
    restarts: int
    relres: float
    history: list = field(default_factory=list)


def gmres(matvec, b: np.ndarray, tol: float = 1e-10, restart: int = 30,
          max_iter: int = 2000, x0: np.ndarray | None = None) -> GmresResult:
    """Restarted GMRES(m) with modified Gram-Schmidt Arnoldi and Givens
    rotations, x0 = 0, no preconditioner (Sec. 5: GMRES, no restart in 1D;
    Sec. 5.3: restart 30).  Stops when the true relative residual
    ||b - A x|| / ||b|| reaches ``tol`` (checked at each restart and when the
    Givens estimate reaches ``tol``)."""
    b = np.asarray(b, dtype=float)
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=float)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return GmresResult(x, 0, 0, 0.0, [0.0])
    hist = []
    total = 0
    restarts = 0
    r = b - matvec(x)
    beta = np.linalg.norm(r)
    hist.append(beta / bn)
    while total < max_iter and beta / bn > tol:
        m = min(restart, max_iter - total)
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            w = matvec(V[j])
            for i in range(j + 1):
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                h0 = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = h0
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bn)
            if abs(g[j + 1]) / bn <= tol or H[j, j] == 0.0:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + V[:j_done].T @ y
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        restarts += 1
    return GmresResult(x, total, restarts, beta / bn, hist)


def arnoldi(matvec, v0: np.ndarray, m: int) -> np.ndarray:
    """m steps of the Arnoldi process (modified Gram-Schmidt, applied twice:
    one pass alone loses orthogonality as the space nears invariance) from
    v0: returns the (k+1) x k upper Hessenberg H with A V_k = V_{k+1} H, k = m
    unless the space became invariant (happy breakdown).  The eigenvalues of
    H[:k, :k] (Ritz values) approximate the spectrum whose clustering Sec. 4
    studies."""
    v0 = np.asarray(v0, dtype=float)
    n = v0.size
    V = np.zeros((m + 1, n))
    H = np.zeros((m + 1, m))
    V[0] = v0 / np.linalg.norm(v0)
    k = 0
    for j in range(m):
        w = matvec(V[j])
        for _ in range(2):
            for i in range(j + 1):
                c = V[i] @ w
                H[i, j] += c
                w = w - c * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        k = j + 1
        if H[j + 1, j] <= 1e-14 * abs(H[: j + 1, j]).max():
            break
        V[j + 1] = w / H[j + 1, j]
    return H[: k + 1, :k]


def solve_gmres(prob: Problem, b: np.ndarray | None = None, tol: float = 1e-13,
                restart: int = 60, max_iter: int = 5000) -> GmresResult:
    """Matrix-free solve of A_N I = b (eq. RT_sys_algebraic) with the oracle's
    own GMRES (Sec. 5)."""
    bb = rhs(prob) if b is None else b
    return gmres(lambda v: apply_A(prob, v), bb, tol=tol, restart=restart, max_iter=max_iter)


def bicgstab(matvec, b: np.ndarray, tol: float = 1e-10, max_iter: int = 5000,
             x0: np.ndarray | None = None) -> GmresResult:
    """BiCGStab (van der Vorst 1992), the paper's second Krylov solver for the
    1D systems (Sec. 5, with GMRES), unpreconditioned, shadow residual = the
    initial residual.  One iteration = two operator applications:
        rho = (r0^, r);  beta = (rho / rho_old) (alpha / omega)
        p = r + beta (p - omega v);  v = A p;  alpha = rho / (r0^, v)
        s = r - alpha v;  t = A s;  omega = (t, s) / (t, t)
        x += alpha p + omega s;  r = s - omega t
    Stops when ||r|| / ||b|| <= tol (recursive residual, confirmed by the true
    residual at exit) or after the half step when ||s|| / ||b|| <= tol.
    ``iterations`` counts full iterations (half steps count as one)."""
    b = np.asarray(b, dtype=float)
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=float)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return GmresResult(x, 0, 0, 0.0, [0.0])
    r = b - matvec(x)
    rhat = r.copy()
    p = np.zeros(n)
    v = np.zeros(n)
    rho_old = alpha = omega = 1.0
    hist = [np.linalg.norm(r) / bn]
    it = 0
    while it < max_iter and hist[-1] > tol:
        rho = rhat @ r
        if rho == 0.0:
            break
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = matvec(p)
        alpha = rho / (rhat @ v)
        s = r - alpha * v
        it += 1
        if np.linalg.norm(s) / bn <= tol:
            x = x + alpha * p
            hist.append(np.linalg.norm(s) / bn)
            break
        t = matvec(s)
        tt = t @ t
        omega = (t @ s) / tt if tt > 0.0 else 0.0
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
        hist.append(np.linalg.norm(r) / bn)
        if omega == 0.0:
            break
    relres = np.linalg.norm(b - matvec(x)) / bn
    return GmresResult(x, it, 0, relres, hist)


def solve_bicgstab(prob: Problem, b: np.ndarray | None = None, tol: float = 1e-13,
                   max_iter: int = 5000) -> GmresResult:
    """Matrix-free solve of A_N I = b (eq. RT_sys_algebraic) with the oracle's
    own BiCGStab (Sec. 5)."""
    bb = rhs(prob) if b is None else b
    return bicgstab(lambda v: apply_A(prob, v), bb, tol=tol, max_iter=max_iter)


# ------------------------------------------------- reduced CRD system (1D only)
def solve_crd_reduced(prob: Problem) -> np.ndarray:
    """Isotropic CRD (Sec. 5.2: P = 1, R = phi phi^T, gamma = (1 - eps)/phi, t = eps B):
    S depends on depth only, S = (1-eps) Jbar + eps B with Jbar = sum w_dir w_nu
    phi I.  Solve (Id - diag(1-eps) Lambda_bar) S = eps B + (1-eps) Jbar_bc with
    Lambda_bar[i, j] = sum_{dir, nu} w w phi Lambda_(dir,nu)[i, j] (N_z x N_z),
    then I = Lambda S + I_in.  Returns I (an independent route to the solution).
    """
    nz, nd, nn = prob.nz, prob.n_dir, prob.n_nu
    phi = prob.R[:, 0] / np.sqrt(prob.R[0, 0])
    phi = phi * np.sign(phi[0])
    one_minus_eps = prob.gamma[:, 0] * phi[0]
    epsB = prob.t_src[:, 0]
    wgt = np.outer(prob.w_dir, prob.w_nu * phi)                  # [nd, nn]
    Lbar = np.zeros((nz, nz))
    for j in range(nz):
        S = np.zeros((nz, nd, nn))
        S[j] = 1.0
        I = lambda_1d(prob, S).reshape(nz, nd, nn)
        Lbar[:, j] = np.einsum("idn,dn->i", I, wgt)
    Ibc = lambda_1d(prob, np.zeros(prob.n), with_inflow=True).reshape(nz, nd, nn)
    Jbc = np.einsum("idn,dn->i", Ibc, wgt)
    M = np.eye(nz) - one_minus_eps[:, None] * Lbar
    S = np.linalg.solve(M, epsB + one_minus_eps * Jbc)
    Sfull = np.broadcast_to(S[:, None, None], (nz, nd, nn)).reshape(-1)
    return lambda_1d(prob, Sfull) + Ibc.reshape(-1)


# ------------------------------------------------------------------ batches
def batch_offsets(probs) -> np.ndarray:
    """Start offsets of each column in the concatenated batch vector (columns
    back to back, each in the ordering of Sec. 3.1)."""
    return np.concatenate([[0], np.cumsum([p.n for p in probs])])


def apply_A_batch(probs, x: np.ndarray) -> np.ndarray:
    """A_N (eq. RT_sys_algebraic) applied column by column to a concatenated
    batch vector."""
    off = batch_offsets(probs)
    return np.concatenate([apply_A(p, x[off[c]:off[c + 1]]) for c, p in enumerate(probs)])


def rhs_batch(probs) -> np.ndarray:
    """b = Lambda_N t + I_in (eq. RT_sys_algebraic) of every column, concatenated."""
    return np.concatenate([rhs(p) for p in probs])


# --------------------------------------------------------------- diagnostics
def cluster_fraction(A: np.ndarray, lo: float = 0.999, hi: float = 1.0 + 1e-12) -> tuple[float, float]:
    """Fraction of eigenvalues with |lambda| in [lo, hi] and min |lambda|
    (the statistic of Tables mono and iso)."""
    lam = np.abs(np.linalg.eigvals(A))
    return float(np.mean((lam >= lo) & (lam <= hi))), float(lam.min())
