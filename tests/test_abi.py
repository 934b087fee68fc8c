"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
entry point include/sfg.h declares, and rejects bad arguments on the host
(no device work is issued by these calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sfg.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sfg_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2010_11254_gb300 import _build
    return ctypes.CDLL(_build.build())


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["sfg_build", "sfg_accel", "sfg_accel_vjp", "sfg_free", "sfg_get_stats", "sfg_get_status",
                     "sfg_status_string", "sfg_default_params", "sfg_export", "sfg_debug_lists"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_host_side_argument_checks(lib):
    import paper_2010_11254_gb300 as sfg
    p = sfg.default_params()
    assert (p.G, p.theta, p.leaf_size, p.group_size, p.quadrupole, p.precision) == (1.0, 0.5, 16, 32, 1, 0)
    lib.sfg_status_string.restype = ctypes.c_char_p
    for code in range(6):
        assert lib.sfg_status_string(code).startswith(b"SFG_")
    lib.sfg_build.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                                      ctypes.c_void_p]
    out = ctypes.c_void_p(1)
    # NULL arrays, n <= 0, n >= 2^31 and bad parameters are rejected before any CUDA call
    assert lib.sfg_build(None, None, None, None, 10, None, None, ctypes.byref(out)) == sfg.SFG_EINVAL
    assert out.value is None
    fake = ctypes.c_void_p(16)
    assert lib.sfg_build(fake, fake, fake, None, 0, None, None, ctypes.byref(out)) == sfg.SFG_EINVAL
    assert lib.sfg_build(fake, fake, fake, None, 1 << 31, None, None, ctypes.byref(out)) == sfg.SFG_EINVAL
    for field, bad in [("leaf_size", 0), ("leaf_size", 257), ("group_size", 33), ("group_size", 0),
                       ("theta", -1.0), ("theta", float("nan")), ("precision", 2), ("quadrupole", 3)]:
        q = sfg.default_params()
        setattr(q, field, bad)
        assert lib.sfg_build(fake, fake, fake, None, 10, ctypes.byref(q), None, ctypes.byref(out)) == sfg.SFG_EINVAL
    lib.sfg_fp32_peak.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.sfg_fp32_peak(None, None, None) == sfg.SFG_EINVAL
    lib.sfg_accel.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p]
    assert lib.sfg_accel(None, None, 1, fake, None, None) == sfg.SFG_EINVAL
