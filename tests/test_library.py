"""The C-ABI library builds, loads and exports every entry point that
include/bg.h declares; host-side argument validation works without a GPU."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bg_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2502_07060_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("bg_plan_create", "bg_plan_destroy", "bg_eval", "bg_workspace_size",
              "bg_plan_describe", "bg_strerror", "bg_last_error", "bg_version"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_2502_07060_gb300 import bg
    assert sorted(bg.EXPORTED) == sorted(n for n in _declared())


def test_strerror_and_version(lib):
    lib.bg_strerror.restype = ctypes.c_char_p
    assert lib.bg_strerror(0) == b"success"
    assert lib.bg_strerror(1) == b"invalid argument"
    assert lib.bg_version() == 3


def _create(lib, n=8, d=6, Ds=6, field=1, p=2147483629, metric=0, S=1, H=1, assign=None):
    h = ctypes.c_void_p()
    lib.bg_plan_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    return lib.bg_plan_create(n, d, Ds, field, p, metric, S, H, assign, ctypes.byref(h))


@pytest.mark.parametrize("kw", [
    dict(n=3), dict(n=13), dict(d=3), dict(d=9), dict(Ds=5), dict(Ds=9),
    dict(p=2147483647 * 2 + 1), dict(p=2147483649), dict(p=4), dict(p=2147483627),  # not prime
    dict(field=3), dict(field=-1), dict(metric=2), dict(field=0, p=7), dict(field=2, p=7), dict(S=0),
    dict(H=0), dict(H=2),
])
def test_plan_rejects_bad_arguments_on_host(lib, kw):
    assert _create(lib, **kw) == 1          # BG_ERR_INVALID_ARG before any CUDA call


def test_eval_rejects_null_plan(lib):
    lib.bg_eval.argtypes = [ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 5 + \
        [ctypes.c_size_t, ctypes.c_void_p]
    assert lib.bg_eval(None, 1, None, None, None, None, None, 0, None) == 1


def test_mixed_plan_rejects_bad_masks_on_host(lib):
    """bg_plan_create_mixed: a four-dimensional-leg mask with bits at or above
    n, and the all-assignment form, are refused before any CUDA call."""
    lib.bg_plan_create_mixed.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p)]
    h = ctypes.c_void_p()
    assert lib.bg_plan_create_mixed(8, 6, 6, 1, 2147483629, 0, 1, 1, None, 1 << 8, ctypes.byref(h)) == 1
    assert lib.bg_plan_create_mixed(5, 6, 6, 1, 2147483629, 0, 1, 1, None, 0xFFFFFFFF, ctypes.byref(h)) == 1
    assert lib.bg_plan_create_mixed(5, 6, 6, 1, 2147483629, 0, 2, 32, None, 0b110, ctypes.byref(h)) == 2
    assert not h.value


def test_fault_injection_arguments(lib):
    """bg_debug_inject_fault validates its site and counts on the host."""
    lib.bg_debug_inject_fault.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    assert lib.bg_debug_inject_fault(0, 0, 1) == 1
    assert lib.bg_debug_inject_fault(4, 0, 1) == 1
    assert lib.bg_debug_inject_fault(2, -1, 1) == 1
    assert lib.bg_debug_inject_fault(2, 0, -1) == 1
    for site in (1, 2, 3):
        assert lib.bg_debug_inject_fault(site, 0, 0) == 0      # disarm


def test_in_place_decision_on_host(lib):
    """The copy-or-in-place decision of the host-buffer paths: its operation
    estimate is the oracle's literal multiplication tally, and at the
    benchmark shape it keeps light F_p batches on copies (they would need
    ~350 GB/s over the host link) and reads complex ones in place (~60 GB/s);
    batches of at most 64 MiB always go in place."""
    from oracle.bg_oracle import op_tally
    from paper_2502_07060_gb300 import bg
    for n, d, Ds in ((4, 4, 4), (5, 4, 4), (8, 6, 6), (8, 4, 6), (10, 6, 8), (12, 8, 8)):
        _, ops = bg.in_place_pays(bg.FIELD_FP, n, d, Ds, 1, 1, 0)
        assert ops == op_tally(n, d, Ds).mul
    E = 1 << 22
    fp_bytes = E * (8 * 6 * 4 * 2 + 4 + 1)
    c64r_bytes = E * (8 * 6 * 8 + 8 * 6 * 16 + 16 + 1)
    assert bg.in_place_pays(bg.FIELD_FP, 8, 6, 6, 1, E, fp_bytes)[0] is False
    assert bg.in_place_pays(bg.FIELD_C64_REAL, 8, 6, 6, 1, E, c64r_bytes)[0] is True
    assert bg.in_place_pays(bg.FIELD_C64, 8, 6, 6, 1, E, E * (8 * 6 * 16 * 2 + 17))[0] is True
    assert bg.in_place_pays(bg.FIELD_C64, 4, 4, 4, 1, E, E * (4 * 4 * 16 * 2 + 17))[0] is False
    assert bg.in_place_pays(bg.FIELD_FP, 8, 6, 6, 1, 1 << 16, 64 << 20)[0] is True
    assert bg.in_place_pays(bg.FIELD_FP, 8, 6, 6, 1, 1 << 16, (64 << 20) + 1)[0] is False
    # all helicities of a point (H amplitudes) carry H times the arithmetic
    assert bg.in_place_pays(bg.FIELD_FP, 10, 4, 4, 1024, 1 << 20, (1 << 20) * 4600)[0] is True
    with pytest.raises(bg.BGError):
        bg.in_place_pays(bg.FIELD_FP, 3, 4, 4, 1, 1, 0)
