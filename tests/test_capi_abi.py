"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/mach.h declares (no device work: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "mach.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(mach_[a-z_0-9]+)\s*\(", hdr)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("mach_sample", "mach_hooi", "mach_core", "mach_error", "mach_sample_free", "mach_strerror"):
        assert n in names


def test_library_builds_and_exports_every_symbol():
    import __graft_entry__ as ge
    ge.build()
    from paper_0909_4969_gb300 import mach
    lib = ctypes.CDLL(mach.LIB_PATH)
    for n in declared_symbols():
        assert hasattr(lib, n), "libmach.so does not export " + n
    # every declared symbol has a binding signature
    for n in declared_symbols():
        assert n in mach.SIGNATURES, "binding lacks " + n


def test_host_only_calls():
    from paper_0909_4969_gb300 import mach
    lib = mach.load()
    assert lib.mach_strerror(1).decode() == "invalid argument"
    assert "sm_103a" in lib.mach_version().decode()
    # argument validation happens before any device work
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(4, 4, 4)
    assert lib.mach_sample(None, 0, 3, dims, 0.5, 1, None, ctypes.byref(h)) == 1
    assert lib.mach_sample(ctypes.c_void_p(16), 0, 5, dims, 0.5, 1, None, ctypes.byref(h)) == 1
    assert lib.mach_sample(ctypes.c_void_p(16), 0, 3, dims, 0.0, 1, None, ctypes.byref(h)) == 1
    assert lib.mach_sample(ctypes.c_void_p(16), 0, 3, dims, 1.5, 1, None, ctypes.byref(h)) == 1
    assert lib.mach_sample(ctypes.c_void_p(17), 0, 3, dims, 0.5, 1, None, ctypes.byref(h)) == 1
    n = ctypes.c_int64()
    assert lib.mach_sample_count(None, ctypes.byref(n)) == 1
    # the bounded-wait self-check validates its poll limit before device work
    assert lib.mach_check_bounded_wait(0, 0, None) == 1
    assert lib.mach_check_bounded_wait((1 << 23) + 1, 1, None) == 1
