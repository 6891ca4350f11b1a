"""GPU parity of the compressed scattering (rt_set_sigma_rank; Sec. 4, Remark
comput) against the oracle's truncated frequency kernel.

The truncation keeps the eigenvalues of W^(1/2) R W^(1/2) above tol * max; it
changes only the float32 operator (mixed apply, inner cycles of the solve).
Bars: the float32 apply against the oracle with the same truncated kernel at
2e-5 (the mixed-apply bar); the solve still reaches the float64 LU solution
to 1e-10 (the float64 operator stays exact).
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2602_21958_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED_APPLY_TOL = 2e-5


@pytest.fixture(scope="module")
def rt():
    from paper_2602_21958_gb300 import build_lib, rt as rtm

    build_lib.build()
    return rtm


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda:0")


def _columns():
    return [W.two_level_column(np.logspace(-3, 3, 13), 4, 2, 40, "r2", 1e-3, 1.0),
            W.two_level_column(np.logspace(-2, 2, 7), 4, 2, 24, "r2", 1e-2, 1.5),
            W.two_level_column(np.logspace(-2, 2, 5), 4, 1, 9, "crd", 1e-2, 1.0)]


def _truncated(cols, tol):
    out, ranks = [], []
    for c in cols:
        Rr, r = O.truncated_frequency_kernel(c, tol)
        out.append(dataclasses.replace(c, R=Rr))
        ranks.append(r)
    return out, ranks


def _far_from_threshold(cols, tol):
    for c in cols:
        sw = np.sqrt(c.w_nu)
        lam = np.abs(np.linalg.eigvalsh(sw[:, None] * c.R * sw[None, :]))
        if np.any(np.abs(lam / lam.max() - tol) < 1e-6 * tol):
            return False
    return True


@pytest.mark.parametrize("tol", [1e-2, 1e-4])
@pytest.mark.parametrize("op", [0, 2])
def test_lowrank_float32_operator_matches_the_oracle(rt, tol, op):
    cols = _columns()
    assert _far_from_threshold(cols, tol)
    tcols, ranks = _truncated(cols, tol)
    h = rt.Handle(cols, n_rhs=2, precision=rt.RT_P_MIXED, max_restart=8)
    rmax = h.rt_set_sigma_rank(tol)
    assert rmax == max(ranks) and rmax < max(c.n_nu for c in cols)
    E = sum(c.n for c in cols)
    x = W.random_vectors(2 * E, 1, 77)[0]
    y = torch.empty(2 * E, dtype=torch.float64, device="cuda:0")
    h.rt_apply(op, dev(x), y)
    torch.cuda.synchronize()
    yc = y.cpu().numpy()
    off = O.batch_offsets(cols)
    for r in range(2):
        for k, (c, tc) in enumerate(zip(cols, tcols)):
            xs = x[r * E + off[k]: r * E + off[k + 1]]
            ref = O.apply_A(tc, xs) if op == 0 else O.sigma_op(tc, xs)
            got = yc[r * E + off[k]: r * E + off[k + 1]]
            assert np.linalg.norm(got - ref) <= MIXED_APPLY_TOL * np.linalg.norm(ref), (tol, op, k, r)
    # the float64 operator of the same handle is untouched
    h.rt_apply(op, dev(x), y, fp64=True)
    torch.cuda.synchronize()
    ref = O.apply_A(cols[0], x[:cols[0].n]) if op == 0 else O.sigma_op(cols[0], x[:cols[0].n])
    assert np.linalg.norm(y.cpu().numpy()[:cols[0].n] - ref) <= 1e-12 * np.linalg.norm(ref)
    # tol = 0 restores the exact kernel
    assert h.rt_set_sigma_rank(0.0) == 0


@pytest.mark.parametrize("n_rhs", [1, 2])
def test_lowrank_inner_cycles_keep_the_solution_exact(rt, n_rhs):
    cols = _columns()
    h = rt.Handle(cols, n_rhs=n_rhs, precision=rt.RT_P_MIXED, max_restart=48)
    h.rt_set_sigma_rank(1e-3)
    E = sum(c.n for c in cols)
    x = torch.zeros(n_rhs * E, dtype=torch.float64, device="cuda:0")
    info = h.rt_solve(None, x, tol=1e-12, tol_inner=1e-2, max_outer=40)
    torch.cuda.synchronize()
    assert info["status"] == rt.RT_OK, info
    ref = np.concatenate([O.solve_dense(c) for c in cols])
    xc = x.cpu().numpy()
    for r in range(n_rhs):
        err = np.linalg.norm(xc[r * E:(r + 1) * E] - ref) / np.linalg.norm(ref)
        assert err <= 1e-10, (r, err, info)


def test_lowrank_is_refused_where_it_does_not_apply(rt):
    p = _columns()[0]
    h64 = rt.Handle(p, precision=rt.RT_P_FP64, max_restart=4)
    with pytest.raises(rt.RTError) as e:
        h64.rt_set_sigma_rank(1e-3)
    assert e.value.code == rt.RT_ERR_ARG
    hm = rt.Handle(p, precision=rt.RT_P_MIXED, max_restart=4)
    with pytest.raises(rt.RTError) as e:
        hm.rt_set_sigma_rank(1.5)
    assert e.value.code == rt.RT_ERR_ARG
