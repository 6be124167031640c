"""CPU-side checks of the C-ABI library: it loads without a GPU, exports every symbol
that include/tenom.h declares, and rejects bad arguments on the host before any CUDA
call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def T():
    import __graft_entry__
    from paper_2010_13289_gb300 import build as B
    B.build()
    from paper_2010_13289_gb300 import tenom
    return tenom


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(tenom_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_symbols()
    for required in ("tenom_create", "tenom_destroy", "tenom_init_state", "tenom_rhs", "tenom_max_dt",
                     "tenom_rk3_step", "tenom_face_dump"):
        assert required in names


def test_library_exports_every_declared_symbol(T):
    L = T.lib()
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_scheme_defaults_on_host(T):
    s = T.make_scheme(6)
    assert s.K == 6 and s.ct_mode == T.CT_CONST and s.ct_const == 1e-5
    assert [s.d[k] for k in range(4)] == [0.45, 0.3, 0.05, 0.2]
    s8 = T.make_scheme(8)
    assert s8.ct_mode == T.CT_ADAPTIVE
    assert abs(sum(s8.d[k] for k in range(6)) - 1.0) < 1e-15
    bad = T.tenom_scheme()
    assert T.lib().tenom_scheme_default(ctypes.byref(bad), 7) == T.TENOM_E_INVALID


@pytest.mark.parametrize("shape,dx,bc,K,lim", [
    ((0,), (0.1,), (0,), 6, 0),          # empty grid
    ((16,), (-0.1,), (0,), 6, 0),        # negative spacing
    ((16,), (0.1,), (5,), 6, 0),         # unknown boundary condition
    ((16,), (0.1,), (0,), 7, 0),         # K not 6 or 8
    ((3,), (0.1,), (0,), 8, 0),          # periodic axis shorter than K/2
    ((16,), (0.1,), (0,), 6, 9),         # unknown limiter
])
def test_create_rejects_bad_arguments(T, shape, dx, bc, K, lim):
    g = T.make_grid(shape, dx, bc)
    s = T.tenom_scheme()
    T.lib().tenom_scheme_default(ctypes.byref(s), 6)
    s.K = K
    s.limiter = lim
    ctx = ctypes.c_void_p()
    st = T.lib().tenom_create(ctypes.byref(ctx), ctypes.byref(g), ctypes.byref(s), None)
    assert st in (T.TENOM_E_INVALID, T.TENOM_E_UNSUPPORTED)
    assert not ctx.value


def test_null_context_calls_fail_cleanly(T):
    L = T.lib()
    assert L.tenom_rhs(None, None, None) == T.TENOM_E_INVALID
    assert L.tenom_destroy(None) == T.TENOM_OK
    assert L.tenom_last_error(None) == b""


def test_positivity_flag_validated_on_host(T):
    """The positivity field takes TENOM_PP_OFF or TENOM_PP_ON; anything else is rejected."""
    g = T.make_grid((16,), (0.1,), (0,))
    s = T.make_scheme(6, positivity=T.PP_ON)
    assert s.positivity == T.PP_ON and T.make_scheme(6).positivity == T.PP_OFF
    s.positivity = 2
    ctx = ctypes.c_void_p()
    assert T.lib().tenom_create(ctypes.byref(ctx), ctypes.byref(g), ctypes.byref(s), None) == T.TENOM_E_INVALID
    assert not ctx.value


def test_batch_create_validates_positivity_on_host(T):
    """tenom_batch_create rejects a positivity flag other than off/on before any CUDA call."""
    import numpy as np
    n = np.array([64, 80], dtype=np.int32)
    dx = np.array([0.01, 0.01])
    s = T.make_scheme(6)
    s.positivity = 7
    b = ctypes.c_void_p()
    st = T.lib().tenom_batch_create(ctypes.byref(b), 2, ctypes.c_void_p(n.ctypes.data),
                                    ctypes.c_void_p(dx.ctypes.data), None, 1.4, ctypes.byref(s), None)
    assert st == T.TENOM_E_INVALID and not b.value
