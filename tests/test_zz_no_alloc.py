"""rt_apply_noalloc: the allocation-free apply (static device scratch) for
callers that cannot allocate device memory at call time -- e.g. code running
while a stream is captured into a CUDA graph, where cudaMalloc is illegal.

Checked through the C ABI against rt_apply (same kernels, handle-owned
scratch) on two calls in a row, so a stale scratch from the first call would
show in the second.  Collected last (file name) so a run that stops at the
first failure has run every other test before it."""
import numpy as np
import pytest

from paper_2602_21958_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 2e-5


@pytest.fixture(scope="module")
def rt():
    from paper_2602_21958_gb300 import build_lib, rt as rtm

    build_lib.build()
    return rtm


def _problems():
    t = np.logspace(-3, 3, 20)
    return [W.two_level_column(t, 4, 2, 12, "r2", 1e-3, 1.0),
            W.two_level_column(t[:9], 6, 1, 7, "crd", 1e-2, 1.0)]


@pytest.mark.parametrize("precision,fp64,tol", [(0, False, FP64_TOL), (1, False, MIXED_TOL), (1, True, FP64_TOL)])
@pytest.mark.parametrize("op", [0, 1, 2, 3])
def test_noalloc_matches_rt_apply_twice(rt, precision, fp64, tol, op):
    probs = _problems()
    h = rt.Handle(probs, n_rhs=2, precision=precision, max_restart=8)
    n = h.length
    for call in range(2):
        x = torch.tensor(W.random_vectors(n, 1, 50 + call)[0], device="cuda:0")
        y_ref = torch.empty_like(x)
        y = torch.full_like(x, float("nan"))
        h.rt_apply(op, x, y_ref, fp64=fp64)
        h.rt_apply_noalloc(op, x, y, fp64=fp64)
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b)


def test_noalloc_rejects_oversized_and_host_buffers(rt):
    big = W.two_level_column(np.logspace(-3, 3, 200), 8, 2, 128, "crd", 1e-3, 1.0)  # 409600 dofs
    h = rt.Handle(big, n_rhs=8, precision=rt.RT_P_FP64, max_restart=4)
    x = torch.zeros(h.length, dtype=torch.float64, device="cuda:0")
    with pytest.raises(rt.RTError) as e:
        h.rt_apply_noalloc(0, x, torch.empty_like(x))
    assert e.value.code == rt.RT_ERR_ARG and "scratch" in str(e.value)
    small = rt.Handle(_problems()[1], precision=rt.RT_P_FP64, max_restart=4)
    xh = np.zeros(small.length)
    with pytest.raises(rt.RTError):
        small.rt_apply_noalloc(0, xh, np.zeros_like(xh))
