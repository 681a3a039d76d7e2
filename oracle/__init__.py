"""Oracle for the Stream-K GEMM -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct CPU code.  Only ``tests/``, the smoke check in
``__graft_entry__`` and the benchmark's CPU-baseline leg may import it.  It
shares no code with the CUDA path (``paper_2407_00044_gb300``) and imports
nothing from it; the CUDA path never imports it.

* ``ref_gemm.c``  -- FP64 triple-loop GEMM and |A||B| scale (plain definition).
* ``schedule.py`` -- Stream-K / DP / hybrid schedule simulator.
* ``fp8.py``      -- E4M3 encode/decode and per-tensor quantisation.

All functions are pinned by ``-m "not gpu"`` tests against closed forms,
invariants, brute force and library routines (see tests/test_oracle_*.py).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build_oracle

_lib = None
_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_int64)


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        L.oracle_gemm_f64.restype = None
        L.oracle_gemm_f64.argtypes = [
            _i64, _i64, _i64,
            _dp, _i64, _i64, _dp, _i64, _i64,
            ctypes.c_double, ctypes.c_double,
            _dp, _i64, _i64, _dp, _i64, _i64, _dp, ctypes.c_int]
        L.oracle_gemm_entries_f64.restype = None
        L.oracle_gemm_entries_f64.argtypes = [
            _i64, _lp, _lp, _i64,
            _dp, _i64, _i64, _dp, _i64, _i64,
            ctypes.c_double, ctypes.c_double,
            _dp, _i64, _i64, _dp, _dp, ctypes.c_int]
        L.oracle_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def to_f64(x) -> np.ndarray:
    """Exact float64 copy of a host tensor/array (bf16, fp16, fp32 and fp8
    values are all exactly representable in float64).  Keeps the logical
    shape; the storage order of the copy is whatever numpy picks, and the
    strides are passed to the C code explicitly."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            x = x.detach().to("cpu")
            if x.dtype in (torch.float8_e4m3fn,):
                raise TypeError("dequantise FP8 codes with oracle.fp8 first")
            return x.to(torch.float64).numpy()
    except ImportError:  # pragma: no cover
        pass
    return np.asarray(x, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _strides(a: np.ndarray):
    s0, s1 = a.strides
    assert s0 % 8 == 0 and s1 % 8 == 0
    return s0 // 8, s1 // 8


def gemm(A, B, alpha: float = 1.0, beta: float = 0.0, C0=None,
         threads: int = 0, want_abs: bool = True):
    """C = alpha * A @ B + beta * C0 and S = |A| @ |B| in FP64.

    Returns (C, S) as float64 arrays of shape (M, N); S is None unless
    ``want_abs``."""
    a, b = to_f64(A), to_f64(B)
    M, K = a.shape
    K2, N = b.shape
    if K != K2:
        raise ValueError("inner dimensions differ")
    C = np.empty((M, N), dtype=np.float64)
    S = np.empty((M, N), dtype=np.float64) if want_abs else None
    c0 = None
    if beta != 0.0:
        c0 = to_f64(C0)
        if c0.shape != (M, N):
            raise ValueError("C0 shape")
    if M == 0 or N == 0:
        return C, S
    a_rs, a_cs = _strides(a)
    b_rs, b_cs = _strides(b)
    c0p, c0_rs, c0_cs = (None, 0, 0)
    if c0 is not None:
        c0p = _ptr(c0)
        c0_rs, c0_cs = _strides(c0)
    lib().oracle_gemm_f64(M, N, K, _ptr(a), a_rs, a_cs, _ptr(b), b_rs, b_cs,
                          float(alpha), float(beta), c0p, c0_rs, c0_cs,
                          _ptr(C), N, 1, _ptr(S) if S is not None else None,
                          int(threads))
    return C, S


def gemm_entries(A, B, rows, cols, alpha: float = 1.0, beta: float = 0.0,
                 C0=None, threads: int = 0):
    """Selected entries (rows[p], cols[p]) of alpha * A @ B + beta * C0, with
    their |A||B| scales.  A and B may be large; only K-length dot products
    are formed."""
    a, b = to_f64(A), to_f64(B)
    M, K = a.shape
    N = b.shape[1]
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    if rows.shape != cols.shape:
        raise ValueError("rows/cols shape")
    if rows.size and (rows.min() < 0 or rows.max() >= M or cols.min() < 0 or cols.max() >= N):
        raise IndexError("entry out of range")
    n = rows.size
    out = np.empty(n, dtype=np.float64)
    s = np.empty(n, dtype=np.float64)
    c0p, c0_rs, c0_cs = (None, 0, 0)
    if beta != 0.0:
        c0 = to_f64(C0)
        c0p = _ptr(c0)
        c0_rs, c0_cs = _strides(c0)
    a_rs, a_cs = _strides(a)
    b_rs, b_cs = _strides(b)
    lib().oracle_gemm_entries_f64(n, rows.ctypes.data_as(_lp), cols.ctypes.data_as(_lp), K,
                                  _ptr(a), a_rs, a_cs, _ptr(b), b_rs, b_cs,
                                  float(alpha), float(beta), c0p, c0_rs, c0_cs,
                                  _ptr(out), _ptr(s), int(threads))
    return out, s


def grad_fp64(A, B, G):
    """Gradient of L = <G, A @ B> (plain definition): dA = G @ B^T,
    dB = A^T @ G, both formed by the FP64 triple loop on transposed views."""
    a, b, g = to_f64(A), to_f64(B), to_f64(G)
    dA, _ = gemm(g, b.T, want_abs=False)
    dB, _ = gemm(a.T, g, want_abs=False)
    return dA, dB


# Normwise acceptance bound (same rounded inputs on both sides):
#   |C - Cref| <= 5e-5 * S + 5e-5 * |beta * C0|            FP32 output
#   |C - Cref| <= 5e-5 * S + 2^-8 * |Cref|                 BF16 output
# the 2^-8 term is the unit roundoff of the final BF16 rounding.
REL_BOUND = 5e-5
BF16_OUT_U = 2.0 ** -8


def bound(S, Cref, out: str = "f32", beta_c0=None):
    tol = REL_BOUND * np.asarray(S, dtype=np.float64)
    if beta_c0 is not None:
        tol = tol + REL_BOUND * np.abs(beta_c0)
    if out == "bf16":
        tol = tol + BF16_OUT_U * np.abs(Cref)
    return tol
