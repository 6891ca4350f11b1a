"""rt_apply_noalloc: the apply entry point that allocates no device memory.

Some callers cannot allocate at call time: a host program that hands the whole
device-memory budget to its own pool at start-up and forbids later
allocations, a real-time loop that must not enter the CUDA allocator (a
cudaMalloc can synchronise the device and take unbounded time), or a plug-in
that runs inside a program owning the device.  For them the source-function
scratch of the apply lives in a fixed-size static device array of the library.

Checked through the C ABI against rt_apply (the same kernels with
handle-owned scratch) bit for bit, on two calls in a row with different
inputs, so a stale scratch from the first call would show in the second: 1D
batches in both precisions, the tensor-core Sigma of a dense-kernel mixed
handle, and a 3D box.  Collected last (file name) so a run that stops at the
first failure has run every other test before it; it also passes alone in a
fresh process."""
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


def _columns():
    t = np.logspace(-3, 3, 20)
    return [W.two_level_column(t, 4, 2, 12, "r2", 1e-3, 1.0),
            W.two_level_column(t[:9], 6, 1, 7, "crd", 1e-2, 1.0)]


def _dense_tc_columns():
    # n_r = 64 and 48 (multiples of 16), column lengths and the batch length
    # multiples of 8: every column runs on the tensor cores
    return [W.two_level_column(np.logspace(-2, 2, 9), 4, 2, 8, "r2", 1e-2, 1.0).with_dense_kernel(),
            W.two_level_column(np.logspace(-3, 1, 7), 4, 2, 6, "r2", 1e-3, 1.0).with_dense_kernel()]


def _box():
    rng = np.random.Generator(np.random.PCG64(7))
    nx, ny, nz, n_nu = 6, 5, 4, 6
    kappa = W.lognormal_opacity((nz, ny, nx), 1.5, rng, kappa0=0.7).ravel()
    dirs, wd = W.level_symmetric(4)
    _, wn, phi, R = W.line_data(n_nu, "r2")
    npts = nx * ny * nz
    return W.Problem(dims=3, nx=nx, ny=ny, nz=nz, z=np.array([1.0, 1.2, 0.9]), dirs=dirs, w_dir=wd, w_nu=wn,
                     chi=kappa[:, None] * phi[None, :], gamma=np.tile((1 - 1e-2) / phi, (npts, 1)),
                     P=W.dipole_3d(dirs), R=R, t_src=np.full((npts, n_nu), 1e-2),
                     I_top=np.zeros(n_nu), I_bot=np.ones(n_nu), formal_solver=W.FS_SCL)


def _twice_bitwise(rt, h, op, fp64, seed):
    """Two rt_apply_noalloc calls in a row, each equal bit for bit to rt_apply
    on the same input; returns the second output."""
    n = h.length
    for call in range(2):
        x = torch.tensor(W.random_vectors(n, 1, seed + call)[0], device="cuda:0")
        y_ref = torch.empty_like(x)
        y = torch.full_like(x, float("nan"))
        h.rt_apply(op, x, y_ref, fp64=fp64)
        h.rt_apply_noalloc(op, x, y, fp64=fp64)
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), (op, call)
        assert np.array_equal(a, b), (op, call, np.abs(a - b).max())
    return x.cpu().numpy(), a


@pytest.mark.parametrize("precision,fp64", [(0, False), (1, False), (1, True)])
@pytest.mark.parametrize("op", [0, 1, 2, 3])
def test_noalloc_columns_bitwise_twice(rt, precision, fp64, op):
    h = rt.Handle(_columns(), n_rhs=2, precision=precision, max_restart=8)
    _twice_bitwise(rt, h, op, fp64, 50)


@pytest.mark.parametrize("op", [0, 2])
def test_noalloc_tensor_core_sigma(rt, op):
    """Dense-kernel mixed handle: Sigma runs on tcgen05 (bf16 operands).  Equal
    to rt_apply bit for bit; the bf16-level difference from the float64
    operator shows that the tensor-core path ran."""
    cols = _dense_tc_columns()
    h = rt.Handle(cols, n_rhs=2, precision=rt.RT_P_MIXED, max_restart=8)
    x, y = _twice_bitwise(rt, h, op, False, 70)
    E = sum(c.n for c in cols)
    f = O.apply_A_batch if op == 0 else (lambda ps, v: np.concatenate(
        [O.sigma_op(p, v[o:o + p.n]) for p, o in zip(ps, O.batch_offsets(ps)[:-1])]))
    ref = np.concatenate([f(cols, x[r * E:(r + 1) * E]) for r in range(2)])
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert 1e-5 < err < 1.5e-2, err


@pytest.mark.parametrize("precision,fp64", [(0, False), (1, False), (1, True)])
@pytest.mark.parametrize("op", [0, 1, 2, 3])
def test_noalloc_box_bitwise_twice(rt, precision, fp64, op):
    h = rt.Handle(_box(), precision=precision, max_restart=4)
    _twice_bitwise(rt, h, op, fp64, 90)


def test_noalloc_rejects_oversized_and_host_buffers(rt):
    big = W.two_level_column(np.logspace(-3, 3, 200), 8, 2, 128, "crd", 1e-3, 1.0)  # 409600 dofs
    h = rt.Handle(big, n_rhs=8, precision=rt.RT_P_FP64, max_restart=4)
    x = torch.zeros(h.length, dtype=torch.float64, device="cuda:0")
    with pytest.raises(rt.RTError) as e:
        h.rt_apply_noalloc(0, x, torch.empty_like(x))
    assert e.value.code == rt.RT_ERR_ARG and "scratch" in str(e.value)
    small = rt.Handle(_columns()[1], precision=rt.RT_P_FP64, max_restart=4)
    xh = np.zeros(small.length)
    with pytest.raises(rt.RTError) as e:
        small.rt_apply_noalloc(0, xh, np.zeros_like(xh))
    assert e.value.code == rt.RT_ERR_ARG
