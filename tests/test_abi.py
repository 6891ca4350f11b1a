"""Host-side checks of the C ABI: the library builds, loads and exports every
function declared in include/*.h (no compute calls without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rt_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2602_21958_gb300 import build_lib, rt

    build_lib.build()
    return rt.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"rt_create", "rt_create_batch", "rt_apply", "rt_solve", "rt_destroy"} <= names
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_error_string(lib):
    from paper_2602_21958_gb300 import rt

    assert "sm_103a" in rt.version()
    assert isinstance(lib.rt_last_error(), bytes)


def test_binding_names_match_abi():
    from paper_2602_21958_gb300 import rt

    assert set(rt.EXPORTS) == _declared()
    assert hasattr(rt.Handle, "rt_apply") and hasattr(rt.Handle, "rt_solve")


def test_missing_library_fails_loudly(tmp_path):
    from paper_2602_21958_gb300 import rt

    with pytest.raises(RuntimeError):
        rt.load(str(tmp_path / "nope.so"))


def test_descriptor_marshalling():
    """rt_desc carries the Problem's sizes, formal solver and array addresses
    (float64, C order); a missing optional array is NULL; an unknown formal
    solver is refused before any call."""
    import dataclasses

    import numpy as np

    from paper_2602_21958_gb300 import rt
    from paper_2602_21958_gb300 import workloads as W

    p = W.two_level_column(np.logspace(-2, 2, 7), 4, 2, 5, "r2", 1e-3, 1.0)
    for fs, code in ((W.FS_SCL, rt.RT_FS_SCL), (W.FS_IE, rt.RT_FS_IE), (W.FS_QSC, rt.RT_FS_QSC),
                     (W.FS_LC, rt.RT_FS_LC)):
        keep = []
        d = rt.make_desc(dataclasses.replace(p, formal_solver=fs), keep)
        assert (d.dims, d.nx, d.ny, d.nz, d.n_dir, d.n_nu) == (1, 1, 1, 7, 8, 5)
        assert d.formal_solver == code
        arrs = keep[0]
        for name in ("z", "dir", "w_dir", "chi", "gamma", "P", "R", "t_src", "I_bot"):
            a = arrs[name]
            assert a.dtype == np.float64 and a.flags.c_contiguous
            assert np.ctypeslib.as_array(getattr(d, name), shape=(a.size,)).tolist() == a.ravel().tolist()
        assert not bool(d.Psi)
    with pytest.raises(ValueError):
        rt.make_desc(dataclasses.replace(p, formal_solver="sc-l"), [])


def test_ritz_values_of_a_full_arnoldi_are_the_eigenvalues():
    """Host half of rt_arnoldi: after n steps on an n x n matrix the square part
    of the Hessenberg matrix carries the whole spectrum (here from the oracle's
    Arnoldi on a non-normal matrix with known distinct eigenvalues)."""
    import numpy as np

    import oracle as O
    from paper_2602_21958_gb300 import rt

    rng = np.random.default_rng(12)
    lam = np.array([0.75, 0.9, 0.99, 1.0, 1.2, 0.5, 0.999, 0.82])
    X = np.eye(8) + 0.2 * rng.standard_normal((8, 8))
    A = X @ np.diag(lam) @ np.linalg.inv(X)
    H = O.arnoldi(lambda v: A @ v, rng.standard_normal(8), 8)
    assert H.shape == (9, 8) or H.shape == (8, 8)
    got = np.sort_complex(rt.ritz_values(H))
    assert np.abs(got - np.sort(lam)).max() < 1e-10


def test_fault_injection_alloc_needs_no_device(monkeypatch):
    """RT_FAULT=alloc: rt_create and rt_create_batch return RT_ERR_OOM before
    any device call (so this runs without a GPU), with a message naming the
    injection; unset, the variable changes nothing."""
    import numpy as np

    from paper_2602_21958_gb300 import rt
    from paper_2602_21958_gb300 import workloads as W

    p = W.two_level_column(np.logspace(-2, 2, 5), 2, 1, 3, "crd", 1e-2, 1.0)
    monkeypatch.setenv("RT_FAULT", "alloc")
    for probs in (p, [p, p]):
        with pytest.raises(rt.RTError) as e:
            rt.Handle(probs)
        assert e.value.code == rt.RT_ERR_OOM and "RT_FAULT=alloc" in str(e.value)
