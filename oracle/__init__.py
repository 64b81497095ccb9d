"""CPU oracle for the particle-particle ladder (TEST INFRASTRUCTURE ONLY).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  The CUDA path never calls it; there is
no CPU fallback.

The arithmetic lives in ``ladder_oracle.c`` (plain FP64 loops, OpenMP over
the virtual index a).  This module compiles it with gcc on first use and
wraps it with ctypes.  See the C file's header for the definition it follows
(Eq. ppl-term, Eq. cholesky, Eq. vfunction-chol) and the fixed summation
orders.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ladder_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libladder_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile the oracle library (gcc, OpenMP) if missing or stale."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, _SRC, "-o", tmp], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d = ctypes.POINTER(ctypes.c_double)
            i = ctypes.POINTER(ctypes.c_int)
            lib.oracle_ladder.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, d, d, d]
            lib.oracle_ladder.restype = ctypes.c_int
            lib.oracle_ladder_pairs.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, d, d,
                                                ctypes.c_int, i, i, d]
            lib.oracle_ladder_pairs.restype = ctypes.c_int
            lib.oracle_eri.argtypes = [ctypes.c_int, ctypes.c_int, d, d]
            lib.oracle_eri.restype = ctypes.c_int
            lib.oracle_ladder_stored.argtypes = [ctypes.c_int, ctypes.c_int, d, d, d]
            lib.oracle_ladder_stored.restype = ctypes.c_int
            lib.oracle_energy.argtypes = [ctypes.c_int, ctypes.c_int, d, d]
            lib.oracle_energy.restype = ctypes.c_double
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(x: np.ndarray):
    assert x.dtype == np.float64 and x.flags.c_contiguous
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def _dims(L: np.ndarray, t2: np.ndarray):
    nchol, nv, nv2 = L.shape
    no, no2, nv3, nv4 = t2.shape
    if not (nv == nv2 == nv3 == nv4 and no == no2):
        raise ValueError("inconsistent shapes")
    return no, nv, nchol


def ladder(L: np.ndarray, t2: np.ndarray, R: np.ndarray | None = None) -> np.ndarray:
    """R + sum_cd (ac|bd) t2[i,j,c,d]; returns a new array (R defaults to zero)."""
    no, nv, nchol = _dims(L, t2)
    out = np.zeros((no, no, nv, nv)) if R is None else np.array(R, dtype=np.float64, copy=True, order="C")
    L = np.ascontiguousarray(L, dtype=np.float64)
    t2 = np.ascontiguousarray(t2, dtype=np.float64)
    rc = _load().oracle_ladder(no, nv, nchol, _dptr(L), _dptr(t2), _dptr(out))
    if rc:
        raise RuntimeError(f"oracle_ladder failed ({rc})")
    return out


def ladder_pairs(L: np.ndarray, t2: np.ndarray, a_list, b_list) -> np.ndarray:
    """Row-subset mode: out[k, i, j] = sum_cd (a_k c|b_k d) t2[i,j,c,d]."""
    no, nv, nchol = _dims(L, t2)
    a = np.ascontiguousarray(a_list, dtype=np.int32)
    b = np.ascontiguousarray(b_list, dtype=np.int32)
    if a.shape != b.shape or a.ndim != 1:
        raise ValueError("a_list and b_list must be 1-D and equal length")
    out = np.zeros((a.size, no, no))
    L = np.ascontiguousarray(L, dtype=np.float64)
    t2 = np.ascontiguousarray(t2, dtype=np.float64)
    ip = ctypes.POINTER(ctypes.c_int)
    rc = _load().oracle_ladder_pairs(no, nv, nchol, _dptr(L), _dptr(t2), int(a.size),
                                     a.ctypes.data_as(ip), b.ctypes.data_as(ip), _dptr(out))
    if rc:
        raise RuntimeError(f"oracle_ladder_pairs failed ({rc})")
    return out


def eri(L: np.ndarray) -> np.ndarray:
    """Stored ERI block V[a,b,c,d] = (ac|bd) = sum_P L[P,a,c] L[P,b,d]."""
    nchol, nv, _ = L.shape
    V = np.zeros((nv, nv, nv, nv))
    L = np.ascontiguousarray(L, dtype=np.float64)
    if _load().oracle_eri(nv, nchol, _dptr(L), _dptr(V)):
        raise RuntimeError("oracle_eri failed")
    return V


def ladder_stored(V: np.ndarray, t2: np.ndarray, R: np.ndarray | None = None) -> np.ndarray:
    """R + sum_cd V[a,b,c,d] t2[i,j,c,d] from a stored ERI block."""
    nv = V.shape[0]
    no = t2.shape[0]
    out = np.zeros((no, no, nv, nv)) if R is None else np.array(R, dtype=np.float64, copy=True, order="C")
    V = np.ascontiguousarray(V, dtype=np.float64)
    t2 = np.ascontiguousarray(t2, dtype=np.float64)
    if _load().oracle_ladder_stored(no, nv, _dptr(V), _dptr(t2), _dptr(out)):
        raise RuntimeError("oracle_ladder_stored failed")
    return out


def energy(t2: np.ndarray, R: np.ndarray) -> float:
    """E_L = sum (2 t2[i,j,a,b] - t2[i,j,b,a]) R[i,j,a,b] (compensated FP64)."""
    no, _, nv, _ = t2.shape
    t2 = np.ascontiguousarray(t2, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    return float(_load().oracle_energy(no, nv, _dptr(t2), _dptr(R)))


def flops_unpacked(no: int, nv: int, nchol: int, npairs: int | None = None) -> float:
    """Multiply-adds x2 the oracle performs: per (a,b) pair 2 X v^2 + 2 o^2 v^2."""
    n = nv * nv if npairs is None else npairs
    return float(n) * (2.0 * nchol * nv * nv + 2.0 * no * no * nv * nv)
