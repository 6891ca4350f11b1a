"""Python binding of the C ABI in include/rt_gb300.h (argument marshalling only).

Every computation runs in librt_gb300.so; this module converts
:class:`paper_2602_21958_gb300.workloads.Problem` objects into ``rt_desc``
structures and tensors/arrays into raw pointers.  It raises if the CUDA library
is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from .workloads import FS_IE, FS_LC, FS_QSC, FS_SCL, Problem

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "librt_gb300.so")

RT_OK, RT_ERR_ARG, RT_ERR_CUDA, RT_ERR_OOM, RT_ERR_NOCONV, RT_ERR_BREAKDOWN, RT_ERR_NONFINITE, \
    RT_ERR_TIMEOUT = range(8)
RT_FS_SCL, RT_FS_IE, RT_FS_QSC, RT_FS_LC = 0, 1, 2, 3
RT_P_FP64, RT_P_MIXED = 0, 1
RT_OP_A, RT_OP_LAMBDA, RT_OP_SIGMA, RT_OP_RHS = 0, 1, 2, 3
RT_KRYLOV_GMRES, RT_KRYLOV_BICGSTAB = 0, 1

_dp = C.POINTER(C.c_double)


class rt_desc(C.Structure):
    _fields_ = [("dims", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("n_dir", C.c_int32), ("n_nu", C.c_int32), ("z", _dp), ("dir", _dp),
                ("w_dir", _dp), ("w_nu", _dp), ("chi", _dp), ("gamma", _dp), ("P", _dp),
                ("R", _dp), ("Psi", _dp), ("t_src", _dp), ("I_top", _dp), ("I_bot", _dp),
                ("formal_solver", C.c_int32)]


class rt_solve_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("tol_inner", C.c_double), ("restart", C.c_int32),
                ("max_outer", C.c_int32), ("use_x0", C.c_int32), ("inner_restart", C.c_int32),
                ("method", C.c_int32), ("max_iter", C.c_int32)]


class rt_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_instances", C.c_int32), ("max_outer", C.c_int32),
                ("max_inner", C.c_int32), ("total_inner", C.c_int64), ("max_relres", C.c_double),
                ("ms", C.c_double), ("bytes", C.c_double), ("inst_outer", C.POINTER(C.c_int32)),
                ("inst_inner", C.POINTER(C.c_int32)), ("inst_relres", _dp)]


EXPORTS = ("rt_create", "rt_create_batch", "rt_vector_length", "rt_apply", "rt_apply_noalloc",
           "rt_autotune", "rt_set_sigma_rank", "rt_tc_timer", "rt_solve", "rt_arnoldi", "rt_destroy",
           "rt_last_error", "rt_version")


class rt_tune_info(C.Structure):
    _fields_ = [("ray_block", C.c_int32), ("ahead", C.c_int32), ("sigma_points", C.c_int32),
                ("from_cache", C.c_int32), ("ms_best", C.c_double), ("ms_default", C.c_double),
                ("box_fb", C.c_int32), ("box_cpt", C.c_int32), ("solve_per_sm", C.c_int32),
                ("solve_inner", C.c_int32), ("solve_ms", C.c_double)]

_lib = None


def load(path: Optional[str] = None) -> C.CDLL:
    """Load librt_gb300.so (raises if it was not built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is missing: build it with __graft_entry__.build()")
    lib = C.CDLL(p)
    vp = C.c_void_p
    lib.rt_create.argtypes = [C.POINTER(rt_desc), C.c_int32, C.c_int32, C.c_int32, C.POINTER(vp)]
    lib.rt_create_batch.argtypes = [C.POINTER(rt_desc), C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                    C.POINTER(vp)]
    lib.rt_vector_length.argtypes = [vp]
    lib.rt_vector_length.restype = C.c_int64
    lib.rt_apply.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp]
    lib.rt_apply_noalloc.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp]
    lib.rt_autotune.argtypes = [vp, C.c_int32, C.POINTER(rt_tune_info), vp]
    lib.rt_autotune.restype = C.c_int
    lib.rt_set_sigma_rank.argtypes = [vp, C.c_double, C.POINTER(C.c_int32)]
    lib.rt_set_sigma_rank.restype = C.c_int
    lib.rt_tc_timer.argtypes = [vp, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    lib.rt_tc_timer.restype = C.c_int
    lib.rt_solve.argtypes = [vp, vp, vp, C.POINTER(rt_solve_opts), C.POINTER(rt_info), vp]
    lib.rt_arnoldi.argtypes = [vp, vp, C.c_int32, vp, C.POINTER(C.c_int32), vp]
    lib.rt_destroy.argtypes = [vp]
    lib.rt_destroy.restype = None
    lib.rt_last_error.restype = C.c_char_p
    lib.rt_version.restype = C.c_char_p
    for name in ("rt_create", "rt_create_batch", "rt_apply", "rt_apply_noalloc", "rt_solve"):
        getattr(lib, name).restype = C.c_int
    if path is None:
        _lib = lib
    return lib


class RTError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rt error {code}: {msg}")
        self.code = code


def _check(code: int):
    if code != RT_OK:
        raise RTError(code, load().rt_last_error().decode())


def _ptr(a) -> C.c_void_p:
    """Raw address of a torch tensor (device or host) or a numpy array."""
    if a is None:
        return C.c_void_p(0)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(a.ctypes.data)
    raise TypeError(type(a))


def _stream_ptr(stream) -> C.c_void_p:
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _as_c(a) -> Optional[np.ndarray]:
    if a is None:
        return None
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def make_desc(p: Problem, keep: list) -> rt_desc:
    """rt_desc for one Problem; arrays are appended to ``keep`` to stay alive."""
    arrs = {
        "z": _as_c(p.z), "dir": _as_c(p.dirs), "w_dir": _as_c(p.w_dir), "w_nu": _as_c(p.w_nu),
        "chi": _as_c(p.chi), "gamma": _as_c(p.gamma), "P": _as_c(p.P), "R": _as_c(p.R),
        "Psi": _as_c(p.Psi), "t_src": _as_c(p.t_src), "I_top": _as_c(p.I_top), "I_bot": _as_c(p.I_bot),
    }
    keep.append(arrs)
    d = rt_desc()
    d.dims, d.nx, d.ny, d.nz = p.dims, p.nx, p.ny, p.nz
    d.n_dir, d.n_nu = p.n_dir, p.n_nu
    for k, v in arrs.items():
        setattr(d, k, v.ctypes.data_as(_dp) if v is not None else _dp())
    fs = {FS_SCL: RT_FS_SCL, FS_IE: RT_FS_IE, FS_QSC: RT_FS_QSC, FS_LC: RT_FS_LC}.get(p.formal_solver)
    if fs is None:
        raise ValueError("unknown formal solver %r" % (p.formal_solver,))
    d.formal_solver = fs
    return d


class Handle:
    """Owner of one rt_handle (a 1D column, a batch of columns, or a 3D box)."""

    def __init__(self, problems: Problem | Sequence[Problem], n_rhs: int = 1,
                 precision: int = RT_P_FP64, max_restart: int = 64):
        lib = load()
        single = isinstance(problems, Problem)
        probs = [problems] if single else list(problems)
        keep: list = []
        h = C.c_void_p()
        if single:
            d = make_desc(probs[0], keep)
            _check(lib.rt_create(C.byref(d), n_rhs, precision, max_restart, C.byref(h)))
        else:
            arr = (rt_desc * len(probs))(*[make_desc(p, keep) for p in probs])
            _check(lib.rt_create_batch(arr, len(probs), n_rhs, precision, max_restart, C.byref(h)))
        self._h = h
        self.problems = probs
        self.n_rhs = n_rhs
        self.precision = precision
        self.max_restart = max_restart
        self.length = int(lib.rt_vector_length(h))

    def close(self):
        if getattr(self, "_h", None):
            load().rt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rt_apply(self, op: int, x, y, fp64: bool = False, stream=None):
        _check(load().rt_apply(self._h, op, int(bool(fp64)), _ptr(x), _ptr(y), _stream_ptr(stream)))

    def rt_apply_noalloc(self, op: int, x, y, fp64: bool = False, stream=None):
        """rt_apply without any allocation: device tensors only, scratch in the
        library's static device array (see include/rt_gb300.h)."""
        _check(load().rt_apply_noalloc(self._h, op, int(bool(fp64)), _ptr(x), _ptr(y), _stream_ptr(stream)))

    def rt_autotune(self, force: bool = False, stream=None, solve: bool = False) -> dict:
        """Time the apply kernels' launch shapes on this problem and keep the
        fastest; with ``solve`` also the persistent mixed solve's CTA shape and
        inner cycle length (batches)."""
        t = rt_tune_info()
        flags = (1 if force else 0) | (2 if solve else 0)
        _check(load().rt_autotune(self._h, flags, C.byref(t), _stream_ptr(stream)))
        return {"ray_block": t.ray_block, "ahead": t.ahead, "sigma_points": t.sigma_points,
                "from_cache": bool(t.from_cache), "ms_best": t.ms_best, "ms_default": t.ms_default,
                "box_fb": t.box_fb, "box_cpt": t.box_cpt, "solve_per_sm": t.solve_per_sm,
                "solve_inner": t.solve_inner, "solve_ms": t.solve_ms}

    def rt_set_sigma_rank(self, tol: float) -> int:
        """Truncate the float32 operator's frequency kernels at ``tol``
        (0: exact); returns the largest rank kept."""
        r = C.c_int32(0)
        _check(load().rt_set_sigma_rank(self._h, float(tol), C.byref(r)))
        return r.value

    def rt_tc_timer(self, on: bool):
        """Start (on) or end a timing session of the tensor-core Sigma kernel;
        ending returns (summed device ms, launches timed)."""
        ms, n = C.c_double(0.0), C.c_int64(0)
        _check(load().rt_tc_timer(self._h, int(bool(on)), C.byref(ms), C.byref(n)))
        return None if on else (ms.value, n.value)

    def rt_solve(self, b, x, tol: float = 1e-11, tol_inner: float = 0.1, restart: Optional[int] = None,
                 max_outer: int = 50, use_x0: bool = False, stream=None, per_instance: bool = False,
                 raise_on_noconv: bool = False, inner_restart: int = 0, method: int = RT_KRYLOV_GMRES,
                 max_iter: int = 0) -> dict:
        o = rt_solve_opts(tol, tol_inner, restart or self.max_restart, max_outer, int(use_x0), inner_restart,
                          method, max_iter)
        info = rt_info()
        n_inst = len(self.problems) * self.n_rhs
        arrs = None
        if per_instance:
            arrs = (np.zeros(n_inst, np.int32), np.zeros(n_inst, np.int32), np.zeros(n_inst))
            info.inst_outer = arrs[0].ctypes.data_as(C.POINTER(C.c_int32))
            info.inst_inner = arrs[1].ctypes.data_as(C.POINTER(C.c_int32))
            info.inst_relres = arrs[2].ctypes.data_as(_dp)
        code = load().rt_solve(self._h, _ptr(b), _ptr(x), C.byref(o), C.byref(info), _stream_ptr(stream))
        # solve outcomes (info filled) are returned; call failures raise
        if code not in (RT_OK, RT_ERR_NOCONV, RT_ERR_BREAKDOWN, RT_ERR_NONFINITE) or \
                (raise_on_noconv and code != RT_OK):
            _check(code)
        out = {"status": code, "max_outer": info.max_outer, "max_inner": info.max_inner,
               "total_inner": info.total_inner, "max_relres": info.max_relres, "ms": info.ms,
               "bytes": info.bytes}
        if arrs is not None:
            out.update(inst_outer=arrs[0], inst_inner=arrs[1], inst_relres=arrs[2])
        return out


    def rt_arnoldi(self, m: int, v0=None, stream=None) -> np.ndarray:
        """m Arnoldi steps on A_N (float64 operator) from v0 (device tensor; None:
        the internal right-hand side); returns the (k+1) x k Hessenberg matrix,
        k the steps taken.  Ritz values: ``ritz_values(H)``."""
        H = np.zeros((m + 1) * m)
        done = C.c_int32(0)
        _check(load().rt_arnoldi(self._h, _ptr(v0), m, H.ctypes.data_as(C.c_void_p), C.byref(done),
                                 _stream_ptr(stream)))
        k = done.value
        return H.reshape(m, m + 1).T[:k + 1, :k].copy()


def ritz_values(H: np.ndarray) -> np.ndarray:
    """Eigenvalues of the square part of an Arnoldi Hessenberg matrix."""
    k = H.shape[1]
    return np.linalg.eigvals(H[:k, :k])


def version() -> str:
    return load().rt_version().decode()
