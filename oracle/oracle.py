"""ctypes front end of the C oracle (``exactsum_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function here
marshals arguments and calls the C code; the arithmetic is all in C.

Functions
---------
exact_sum(bits, in_dtype, out_dtype, mode, threads)
    Exact sum of the elements (given as an unsigned-integer bit array), rounded
    once; returns the result's bit pattern as a Python int.
exact_sum_segmented(bits, offsets, in_dtype, out_dtype, mode, threads)
    The same per CSR segment; returns a numpy bit array.
exact_value(bits, in_dtype)
    The exact sum as a Python int in units of the input format's smallest
    subnormal (non-finite elements skipped).
round_value(value, unit_exp, out_dtype, mode)
    Round the exact value ``value * 2**unit_exp`` (value a Python int).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

F64, F32, BF16 = 0, 1, 2
RNE, RTZ, RUP, RDOWN = 0, 1, 2, 3
_WIDTH = {F64: 8, F32: 4, BF16: 2}
_NP = {F64: np.uint64, F32: np.uint32, BF16: np.uint16}
_LIMBS = 96

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "exactsum_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only) and return its path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.oracle_sum.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
            lib.oracle_sum.restype = ctypes.c_int
            lib.oracle_segmented_sum.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                 ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_void_p]
            lib.oracle_segmented_sum.restype = ctypes.c_int
            lib.oracle_exact_limbs.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                               ctypes.c_void_p]
            lib.oracle_exact_limbs.restype = ctypes.c_int
            lib.oracle_round_limbs.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_void_p]
            lib.oracle_round_limbs.restype = ctypes.c_int
            _lib = lib
    return _lib


def _as_bits(bits, dtype):
    a = np.ascontiguousarray(bits)
    if a.dtype.itemsize != _WIDTH[dtype]:
        raise TypeError(f"expected {_WIDTH[dtype]}-byte elements, got {a.dtype}")
    return a


def exact_sum(bits, in_dtype: int = F64, out_dtype: int | None = None, mode: int = RNE,
              threads: int = 1) -> int:
    lib = _load()
    out_dtype = in_dtype if out_dtype is None else out_dtype
    a = _as_bits(bits, in_dtype)
    res = np.zeros(1, dtype=_NP[out_dtype])
    rc = lib.oracle_sum(a.ctypes.data if a.size else None, a.size, in_dtype, out_dtype, mode,
                        threads, res.ctypes.data)
    if rc:
        raise ValueError("oracle_sum rejected its arguments")
    return int(res[0])


def exact_sum_segmented(bits, offsets, in_dtype: int = F64, out_dtype: int | None = None,
                        mode: int = RNE, threads: int = 1) -> np.ndarray:
    lib = _load()
    out_dtype = in_dtype if out_dtype is None else out_dtype
    a = _as_bits(bits, in_dtype)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    S = len(off) - 1
    res = np.zeros(max(S, 1), dtype=_NP[out_dtype])
    rc = lib.oracle_segmented_sum(a.ctypes.data if a.size else None, off.ctypes.data, S,
                                  in_dtype, out_dtype, mode, threads, res.ctypes.data)
    if rc:
        raise ValueError("oracle_segmented_sum rejected its arguments")
    return res[:S]


def exact_value(bits, in_dtype: int = F64) -> int:
    lib = _load()
    a = _as_bits(bits, in_dtype)
    limbs = np.zeros(_LIMBS, dtype=np.uint32)
    rc = lib.oracle_exact_limbs(a.ctypes.data if a.size else None, a.size, in_dtype,
                                limbs.ctypes.data)
    if rc < 0:
        raise ValueError("oracle_exact_limbs rejected its arguments")
    v = int.from_bytes(limbs.tobytes(), "little")
    if v >> (32 * _LIMBS - 1):
        v -= 1 << (32 * _LIMBS)
    return v


def round_value(value: int, unit_exp: int, out_dtype: int = F64, mode: int = RNE) -> int:
    lib = _load()
    sign = 1 if value < 0 else 0
    mag = -value if sign else value
    if mag.bit_length() > 32 * _LIMBS - 1:
        raise ValueError("value too large for the oracle")
    limbs = np.frombuffer(mag.to_bytes(4 * _LIMBS, "little"), dtype=np.uint32).copy()
    res = np.zeros(1, dtype=_NP[out_dtype])
    rc = lib.oracle_round_limbs(limbs.ctypes.data, _LIMBS, sign, unit_exp, out_dtype, mode,
                                res.ctypes.data)
    if rc:
        raise ValueError("oracle_round_limbs rejected its arguments")
    return int(res[0])
