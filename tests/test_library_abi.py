"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
symbol that include/ffb.h declares, and rejects invalid arguments before any
device work (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1412_0781_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def _declared():
    txt = open(os.path.join(ROOT, "include", "ffb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ffb_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("ffb_plan", "ffb_expand", "ffb_covariance", "ffb_eig", "ffb_denoise",
                     "ffb_expand_adjoint", "ffb_plan_destroy", "ffb_strerror", "ffb_cov_get"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_1412_0781_gb300 import ffb
    assert sorted(ffb.SIGNATURES) == _declared()


def test_library_is_built_for_sm_103a(lib):
    from paper_1412_0781_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_strerror(lib):
    lib.ffb_strerror.restype = ctypes.c_char_p
    assert lib.ffb_strerror(0) == b"ok"
    assert lib.ffb_strerror(-1) == b"invalid argument"
    assert lib.ffb_strerror(12345) == b"unknown status"


@pytest.mark.parametrize("L,c,R,eps,prec", [
    (4, 0.5, 2.0, 1e-6, 0),      # L too small
    (64, 0.6, 32.0, 1e-6, 0),    # c > 1/2
    (64, 0.5, 33.0, 1e-6, 0),    # R > L/2
    (64, 0.5, 0.0, 1e-6, 0),     # R <= 0
    (64, 0.5, 32.0, 1e-9, 0),    # eps below float32 reach
    (64, 0.5, 32.0, 1e-6, 7),    # unknown precision
])
def test_plan_rejects_bad_arguments(lib, L, c, R, eps, prec):
    h = ctypes.c_void_p()
    lib.ffb_plan.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_double,
                             ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_void_p]
    assert lib.ffb_plan(ctypes.byref(h), L, c, R, eps, prec, None) == -1
    assert not h.value


def test_null_plan_is_rejected(lib):
    lib.ffb_expand.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                               ctypes.c_void_p]
    assert lib.ffb_expand(None, None, 1, None, None) == -1
    assert lib.ffb_plan_destroy(None) == 0


def test_group_calls_reject_bad_arguments(lib):
    vp = ctypes.c_void_p
    lib.ffb_group_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp), vp]
    h = vp()
    plans = (vp * 2)(None, None)
    assert lib.ffb_group_create(ctypes.byref(h), 0, plans, None) == -1     # S < 1
    assert lib.ffb_group_create(ctypes.byref(h), 65, plans, None) == -1    # S > 64
    assert lib.ffb_group_create(ctypes.byref(h), 2, plans, None) == -1     # NULL plans
    assert not h.value
    lib.ffb_group_expand_cov.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(vp), ctypes.c_int, vp]
    assert lib.ffb_group_expand_cov(None, None, None, None, 1, None) == -1
    lib.ffb_group_covariance.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int64), ctypes.c_int, vp]
    assert lib.ffb_group_covariance(None, None, None, 1, None) == -1
    lib.ffb_group_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    assert lib.ffb_group_info(None, None) == -1
    assert lib.ffb_group_destroy(None) == 0
