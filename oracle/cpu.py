"""ctypes loader for ``cpu_ntt.c`` (the C statement of the transform).

TEST INFRASTRUCTURE: see ``oracle/__init__.py`` for who may call this.
The shared library is built in-tree by ``build()`` below (plain gcc, no CUDA).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import field as fld

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpu_ntt.c")
_LIB = os.path.join(_HERE, "libcpu_ntt.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-Wall", "-Wextra", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.zo_ntt.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u32p, u32p, u32p, ctypes.c_int]
        L.zo_eval.argtypes = [ctypes.c_int, ctypes.c_uint64, u32p, u32p, u32p]
        L.zo_groth16_h.argtypes = [ctypes.c_int, ctypes.c_int, u32p, u32p, u32p, u32p, ctypes.c_int]
        L.zo_root.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u32p]
        L.zo_mont_mul.argtypes = [ctypes.c_int, u32p, u32p, u32p]
        L.zo_two_adicity.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _fid(F) -> int:
    return fld.FIELD_IDS[fld.get(F).name]


def _limbs(v: int) -> np.ndarray:
    return np.frombuffer(int(v).to_bytes(32, "little"), dtype=np.uint32).copy()


def threads_default() -> int:
    return int(lib().zo_threads_default())


def ntt(F, X: np.ndarray, inverse: bool = False, shift_mont: int | None = None,
        threads: int | None = None) -> np.ndarray:
    """Montgomery-form limbs [n, 8] -> transform, same layout: the C oracle's
    radix-2 transform (Section II-B; inverse with n^-1, coset with shift^j,
    as in ntt_ref.ntt)."""
    X = np.ascontiguousarray(X, dtype=np.uint32)
    n = X.shape[0]
    L = n.bit_length() - 1
    out = np.empty_like(X)
    sh = None if shift_mont is None else _limbs(shift_mont)
    rc = lib().zo_ntt(_fid(F), L, int(inverse), None if sh is None else _p(sh), _p(X), _p(out),
                      threads or threads_default())
    if rc:
        raise RuntimeError(f"zo_ntt failed ({rc})")
    return out


def eval_at(F, coeffs: np.ndarray, x_mont: int) -> int:
    """sum_j c_j x^j with every value in Montgomery form (one output of the
    Section II-B definition when x = w^k); returns an int."""
    coeffs = np.ascontiguousarray(coeffs, dtype=np.uint32)
    xs = _limbs(x_mont)
    out = np.zeros(8, dtype=np.uint32)
    rc = lib().zo_eval(_fid(F), coeffs.shape[0], _p(coeffs), _p(xs), _p(out))
    if rc:
        raise RuntimeError("zo_eval failed")
    return int.from_bytes(out.tobytes(), "little")


def groth16_h(F, A, B, C, threads: int | None = None) -> np.ndarray:
    """The Groth16 H sequence of Fig. 2 (Section IV-A) in the C oracle, on
    Montgomery-form limbs."""
    A, B, C = (np.ascontiguousarray(v, dtype=np.uint32) for v in (A, B, C))
    n = A.shape[0]
    out = np.empty_like(A)
    rc = lib().zo_groth16_h(_fid(F), n.bit_length() - 1, _p(A), _p(B), _p(C), _p(out),
                            threads or threads_default())
    if rc:
        raise RuntimeError("zo_groth16_h failed")
    return out


def root(F, log_n: int, inverse: bool = False) -> int:
    """The C oracle's primitive 2^log_n-th root (Section II-B), Montgomery form."""
    out = np.zeros(8, dtype=np.uint32)
    if lib().zo_root(_fid(F), log_n, int(inverse), _p(out)):
        raise ValueError("bad root request")
    return int.from_bytes(out.tobytes(), "little")


def mont_mul(F, a: int, b: int) -> int:
    """The C oracle's Montgomery product a b 2^-256 mod r (FF_mul, Section IV-B)."""
    out = np.zeros(8, dtype=np.uint32)
    lib().zo_mont_mul(_fid(F), _p(_limbs(a)), _p(_limbs(b)), _p(out))
    return int.from_bytes(out.tobytes(), "little")


def two_adicity(F) -> int:
    """The C oracle's 2-adicity of r - 1."""
    return int(lib().zo_two_adicity(_fid(F)))
