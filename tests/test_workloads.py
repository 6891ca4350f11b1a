"""Checks of the seeded input generators (quadratures, profiles, kernels)."""
import math

import numpy as np
import pytest

from paper_2602_21958_gb300 import workloads as W


def test_gauss_legendre_moments():
    d, w = W.gauss_legendre_directions(8, 2)
    mu = d[:, 2]
    assert abs(w.sum() - 1) < 1e-15
    for k in range(0, 8):  # n/2 = 4 nodes per hemisphere: exact to degree 7 on each
        ref = 1.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * mu ** k) - ref) < 1e-14
    assert np.all(np.diff(mu) >= 0) and np.all(mu[:8] < 0)
    assert np.allclose(np.linalg.norm(d, axis=1), 1)


@pytest.mark.parametrize("order,count", [(4, 24), (6, 48), (8, 80)])
def test_level_symmetric_moments(order, count):
    d, w = W.level_symmetric(order)
    assert d.shape == (count, 3) and np.all(w > 0)
    assert np.allclose(np.linalg.norm(d, axis=1), 1, atol=1e-7)
    assert abs(w.sum() - 1) < 1e-14
    for ax in range(3):
        assert abs(np.sum(w * d[:, ax] ** 2) - 1 / 3) < 1e-7
        assert abs(np.sum(w * d[:, ax] ** 4) - 1 / 5) < 1e-7
        assert abs(np.sum(w * d[:, ax])) < 1e-15
    assert np.all(np.diff(d[:, 2]) >= 0)


def test_voigt_against_direct_convolution():
    from scipy.integrate import quad

    a = 0.05
    for x in (0.0, 0.8, 2.5, 6.0):
        f = lambda y: math.exp(-y * y) / ((x - y) ** 2 + a * a)
        val = quad(f, -np.inf, np.inf, points=None, limit=400, epsabs=1e-14, epsrel=1e-12)[0]
        ref = a / math.pi ** 1.5 * val
        assert abs(W.voigt(np.array([x]), a)[0] / ref - 1) < 1e-9


def test_r2a_small_damping_limit():
    """a -> 0: R_II-A(x, x') -> erfc(max(|x|,|x'|)) / 2."""
    from scipy.special import erfc

    x = np.linspace(-3, 3, 13)
    R = W.redistribution_r2a(x, 1e-7)
    ref = 0.5 * erfc(np.maximum(np.abs(x)[:, None], np.abs(x)[None, :]))
    assert np.abs(R - ref).max() < 1e-5


@pytest.mark.parametrize("kind", ["r2", "r3"])
def test_redistribution_marginal_is_profile(kind):
    """int R(x, x') dx' = phi(x) (normalisation of R_II-A and R_III-A)."""
    a = 0.05
    tail = np.logspace(np.log10(11.5), np.log10(4000.0), 300)
    xf = np.concatenate([-tail[::-1], np.linspace(-11, 11, 4401), tail])
    wf = W.trapezoid_weights(xf)
    xs = np.array([0.0, 0.9, 2.2])
    fn = W.r2a_pairs if kind == "r2" else W.r3a_pairs
    R = fn(np.repeat(xs, len(xf)), np.tile(xf, len(xs)), a).reshape(len(xs), len(xf))
    assert np.allclose(R @ wf, W.voigt(xs, a), rtol=2e-3)
    Rt = fn(np.tile(xf, len(xs)), np.repeat(xs, len(xf)), a).reshape(len(xs), len(xf))
    assert np.allclose(R, Rt, rtol=1e-13, atol=1e-16)


def test_conservative_rescaling():
    x, w, phi, R = W.line_data(40, "r23")
    assert np.allclose(R @ w, phi, rtol=1e-13) and np.allclose(R, R.T, atol=1e-17)
    assert abs(np.sum(w * phi) - 1) < 1e-14


def test_lognormal_field_statistics():
    rng = np.random.Generator(np.random.PCG64(7))
    k = W.lognormal_opacity((32, 32, 32), 4.0, rng)
    g = np.log(k) + 0.5
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1) < 1e-12


def test_configs_shapes():
    c1 = W.config_c1()
    assert c1.n == 10752
    c2 = W.config_c2()
    assert c2.n == 131072
    cols = W.config_c5(n_col=6)
    assert all(64 <= c.nz <= 512 and 32 <= c.n_nu <= 128 and c.n_dir == 16 for c in cols)
    c3 = W.config_c3(n=8)
    assert c3.n == 8 ** 3 * 48 * 32


def test_trapezoid_weights_exact_for_linear_functions_on_uneven_grids():
    x = np.array([-2.0, -1.7, -0.2, 0.1, 1.5, 4.0])
    w = W.trapezoid_weights(x)
    assert abs(w.sum() - 6.0) < 1e-15                       # int 1 dx
    assert abs(np.sum(w * x) - 0.5 * (16.0 - 4.0)) < 1e-14  # int x dx


def test_mono_legendre_coefficients_are_the_printed_ones():
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    assert list(W.MONO_LEGENDRE) == gold["mono_legendre"]["d"]


def test_azimuth_averaged_dipole():
    """1 + P2(mu) P2(mu') / 2 is the average over the azimuth difference of the
    dipole phase 3/4 (1 + cos^2 Theta), cos Theta = mu mu' + s s' cos(dphi):
    checked by an equispaced azimuth rule (exact for this degree-2 trig polynomial)."""
    mu = np.array([-0.93, -0.4, 0.05, 0.61, 0.99])
    s = np.sqrt(1 - mu * mu)
    dphi = 2 * np.pi * np.arange(16) / 16
    c = mu[:, None, None] * mu[None, :, None] + s[:, None, None] * s[None, :, None] * np.cos(dphi)
    avg = np.mean(0.75 * (1 + c * c), axis=-1)
    assert np.abs(W.dipole_azimuth_averaged(mu) - avg).max() < 1e-14
    # the 3D dipole over the same direction pairs, averaged the same way
    for i in range(len(mu)):
        for j in range(len(mu)):
            d = np.array([[s[i], 0.0, mu[i]]] + [[s[j] * np.cos(p), s[j] * np.sin(p), mu[j]] for p in dphi])
            assert abs(np.mean(W.dipole_3d(d)[0, 1:]) - avg[i, j]) < 1e-14
