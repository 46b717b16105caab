"""ctypes binding of the C oracle (``oracle/bg_oracle.c``).

TEST INFRASTRUCTURE ONLY (see ``oracle/bg_oracle.c``).  ``build()`` compiles
the C file with gcc and OpenMP into ``oracle/_build/``; nothing here touches
the CUDA library.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bg_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libbg_oracle.so")
_lib = None


def build(force=False):
    """Compile the C oracle (-O3 without host-specific flags, so the x86 and
    Arm builds give the same results; no floating-point contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=gnu11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", _SRC,
           "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        f64p = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.bgo_amp_fp.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint32,
                                   ctypes.c_int, ctypes.c_int64, u32p, u32p, u32p, u8p, ctypes.c_int]
        lib.bgo_amp_fp.restype = ctypes.c_int
        lib.bgo_amp_c64.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int64, f64p, f64p, f64p, u8p, ctypes.c_int]
        lib.bgo_amp_c64.restype = ctypes.c_int
        lib.bgo_amp_c64dd.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int64, f64p, f64p, f64p, u8p, ctypes.c_int]
        lib.bgo_amp_c64dd.restype = ctypes.c_int
        lib.bgo_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def max_threads():
    return _load().bgo_max_threads()


def amp_fp(k, eps, p, metric=0, nthreads=0):
    """Amplitudes over F_p.  k: uint32 [E][n][d], eps: uint32 [E][n][Ds]
    (canonical residues).  Returns (out uint32 [E], status uint8 [E])."""
    lib = _load()
    k = np.ascontiguousarray(k, dtype=np.uint32)
    eps = np.ascontiguousarray(eps, dtype=np.uint32)
    E, n, d = k.shape
    Ds = eps.shape[2]
    if eps.shape[:2] != (E, n):
        raise ValueError("eps shape does not match k")
    out = np.zeros(E, dtype=np.uint32)
    st = np.zeros(E, dtype=np.uint8)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    rc = lib.bgo_amp_fp(n, d, Ds, p, metric, E,
                        k.ctypes.data_as(u32p), eps.ctypes.data_as(u32p),
                        out.ctypes.data_as(u32p), st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                        nthreads)
    if rc != 0:
        raise ValueError("C oracle rejected its arguments")
    return out, st


def amp_c64(k, eps, metric=0, nthreads=0):
    """Amplitudes over complex FP64.  k: complex128 [E][n][d], eps: complex128
    [E][n][Ds].  Returns (out complex128 [E], status uint8 [E])."""
    lib = _load()
    k = np.ascontiguousarray(k, dtype=np.complex128)
    eps = np.ascontiguousarray(eps, dtype=np.complex128)
    E, n, d = k.shape
    Ds = eps.shape[2]
    if eps.shape[:2] != (E, n):
        raise ValueError("eps shape does not match k")
    out = np.zeros(E, dtype=np.complex128)
    st = np.zeros(E, dtype=np.uint8)
    f64p = ctypes.POINTER(ctypes.c_double)
    rc = lib.bgo_amp_c64(n, d, Ds, metric, E,
                         k.ctypes.data_as(f64p), eps.ctypes.data_as(f64p),
                         out.ctypes.data_as(f64p), st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                         nthreads)
    if rc != 0:
        raise ValueError("C oracle rejected its arguments")
    return out, st


def amp_c64dd(k, eps, metric=0, nthreads=0):
    """Double-double evaluation of the complex amplitudes.  Returns (hi
    complex128 [E], lo complex128 [E], status uint8 [E]) with the value
    hi + lo to about 106 bits."""
    lib = _load()
    k = np.ascontiguousarray(k, dtype=np.complex128)
    eps = np.ascontiguousarray(eps, dtype=np.complex128)
    E, n, d = k.shape
    Ds = eps.shape[2]
    if eps.shape[:2] != (E, n):
        raise ValueError("eps shape does not match k")
    out = np.zeros((E, 4), dtype=np.float64)
    st = np.zeros(E, dtype=np.uint8)
    f64p = ctypes.POINTER(ctypes.c_double)
    rc = lib.bgo_amp_c64dd(n, d, Ds, metric, E,
                           k.ctypes.data_as(f64p), eps.ctypes.data_as(f64p),
                           out.ctypes.data_as(f64p), st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                           nthreads)
    if rc != 0:
        raise ValueError("C oracle rejected its arguments")
    hi = out[:, 0] + 1j * out[:, 2]
    lo = out[:, 1] + 1j * out[:, 3]
    return hi, lo, st
