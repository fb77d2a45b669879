"""Host-only checks of the C ABI: the library loads without a GPU, exports every entry point
declared in include/p3m.h, fills default parameters and refuses bad parameters before any
device call."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "p3m.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:p3m_status|const char\*)\s+(p3m_\w+)\s*\(", text,
                                 flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2103_02046_gb300 import build as b
    if not os.path.exists(b.LIB):
        if shutil.which(b.nvcc()) is None and not os.path.exists(b.nvcc()):
            pytest.skip("nvcc not available to build the library")
        b.build()
    from paper_2103_02046_gb300 import p3m
    return p3m.lib()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("p3m_create", "p3m_deposit", "p3m_solve", "p3m_forces", "p3m_push",
                     "p3m_backward", "p3m_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_default_params(lib):
    from paper_2103_02046_gb300 import p3m
    p = p3m.default_params()
    assert tuple(p.n) == (64, 64, 64)
    assert p.assign_order == 2 and p.rc_over_h == 2.0 and p.kappa == 3.0
    assert p.precision == p3m.FP64 and p.pm_bc == 0 and p.pp_bc == 0
    assert p.mass == pytest.approx(1e-15 / 1.602176634e-19 * 9.1093837015e-31, rel=1e-15)


def test_create_refuses_bad_params_without_touching_the_device(lib):
    from paper_2103_02046_gb300 import p3m
    h = ctypes.c_void_p()
    for bad in (dict(n=(4, 16, 16)), dict(assign_order=0), dict(h=(1e-5, -1.0, 1e-5)),
                dict(precision=2), dict(q=0.0), dict(mass=0.0), dict(deterministic=2),
                dict(deterministic=1, precision=p3m.FP32_MIXED),
                dict(deterministic=1, pm_bc=2), dict(adj_slots=2, adj_segment=0),
                dict(search_rows=4), dict(search_rows=-1), dict(search_xcells=3),
                dict(search_xcells=64),
                # an explicit search layout over the cell budget (max(4 n_max, 2^20) cells)
                dict(n=(512, 512, 512), search_rows=3, search_xcells=32),
                dict(n=(512, 512, 512), search_xcells=32)):
        cp = p3m.Params(**bad).to_c()
        assert lib.p3m_create(ctypes.byref(cp), 10, None, ctypes.byref(h)) == p3m.P3M_EINVAL
        assert not h.value
    cp = p3m.Params().to_c()
    assert lib.p3m_create(ctypes.byref(cp), 0, None, ctypes.byref(h)) == p3m.P3M_EINVAL
    assert lib.p3m_create(None, 10, None, ctypes.byref(h)) == p3m.P3M_EINVAL
    assert lib.p3m_destroy(None) == p3m.P3M_OK
    assert lib.p3m_last_error(None) == b"null context"


def test_counts_refuse_null_arguments(lib):
    from paper_2103_02046_gb300 import p3m
    v = ctypes.c_int64(-1)
    lib.p3m_pair_count.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int64)]
    assert lib.p3m_pair_count(None, ctypes.byref(v), None) == p3m.P3M_EINVAL
    assert lib.p3m_candidate_count(None, ctypes.byref(v)) == p3m.P3M_EINVAL
    assert v.value == -1
