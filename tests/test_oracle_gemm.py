"""Pins for the FP64 oracle GEMM (CPU only).

Each check compares the oracle with something other than itself: a closed
form, an exact small-integer identity, numpy's independent FP64 matmul, or
the paper's own printed numbers.  The closed forms use non-symmetric
operands, so a transposed operand, a swapped index, a dropped term or a
wrong sign changes the answer.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import workloads

HERE = os.path.dirname(os.path.abspath(__file__))


def _closed_form_operands(M, N, K):
    i = np.arange(M, dtype=np.float64)[:, None]
    k = np.arange(K, dtype=np.float64)[None, :]
    A = i + 2.0 * k + 1.0                        # M x K
    kk = np.arange(K, dtype=np.float64)[:, None]
    j = np.arange(N, dtype=np.float64)[None, :]
    B = (kk + 1.0) * (j - 3.0)                   # K x N
    # sum_k (i + 2k + 1)(k + 1)(j - 3) = (j - 3) * ((i + 1) * s1 + 2 * s2)
    s1 = K * (K + 1) / 2.0                       # sum_{k<K} (k + 1)
    s2 = (K - 1) * K * (2 * K - 1) / 6.0 + (K - 1) * K / 2.0   # sum k(k+1)
    C = (j - 3.0) * ((i + 1.0) * s1 + 2.0 * s2)
    return A, B, C


@pytest.mark.parametrize("a_order,b_order", [("C", "C"), ("F", "C"), ("C", "F"), ("F", "F")])
@pytest.mark.parametrize("shape", [(5, 7, 3), (17, 9, 33), (1, 1, 1), (64, 3, 130)])
def test_closed_form_any_storage_order(shape, a_order, b_order):
    M, N, K = shape
    A, B, Cx = _closed_form_operands(M, N, K)
    A = np.asarray(A, order=a_order)
    B = np.asarray(B, order=b_order)
    C, S = oracle.gemm(A, B)
    assert np.array_equal(C, Cx)          # integers far below 2^53: exact
    # Operands are non-negative except (j - 3), so S = |C|.
    assert np.array_equal(S, np.abs(Cx))


def test_transposed_views():
    M, N, K = 6, 5, 4
    A, B, Cx = _closed_form_operands(M, N, K)
    # Pass A and B as transposed views of their transposes.
    C, _ = oracle.gemm(np.ascontiguousarray(A.T).T, np.ascontiguousarray(B.T).T)
    assert np.array_equal(C, Cx)
    # C^T = B^T A^T
    Ct, _ = oracle.gemm(B.T, A.T)
    assert np.array_equal(Ct, Cx.T)


def test_identity_alpha_beta():
    K = 24
    B = workloads.small_int((K, 13), seed=3).numpy()
    C0 = workloads.small_int((K, 13), seed=4).numpy()
    I = np.eye(K)
    C, _ = oracle.gemm(I, B, alpha=2.0, beta=-0.5, C0=C0)
    assert np.array_equal(C, 2.0 * B - 0.5 * C0)
    # alpha = 0: only the beta term
    C, _ = oracle.gemm(I, B, alpha=0.0, beta=3.0, C0=C0)
    assert np.array_equal(C, 3.0 * C0)


def test_rank_one():
    M, N, K = 19, 23, 37
    u = workloads.small_int((M,), seed=5).numpy().astype(np.float64)
    v = workloads.small_int((N,), seed=6).numpy().astype(np.float64)
    A = np.repeat(u[:, None], K, axis=1)
    B = np.repeat(v[None, :], K, axis=0)
    C, S = oracle.gemm(A, B)
    assert np.array_equal(C, K * np.outer(u, v))
    assert np.array_equal(S, K * np.outer(np.abs(u), np.abs(v)))


def test_abs_scale_alternating_signs():
    M, N, K = 7, 6, 11
    i = np.arange(M)[:, None]
    k = np.arange(K)[None, :]
    A = ((-1.0) ** (i + k)) * (i + 1.0)
    kk = np.arange(K)[:, None]
    j = np.arange(N)[None, :]
    B = ((-1.0) ** kk) * (j + 1.0)
    C, S = oracle.gemm(A, B)
    sign_i = (-1.0) ** np.arange(M)[:, None]
    assert np.array_equal(C, K * sign_i * (i + 1.0) * (j + 1.0))
    assert np.array_equal(S, K * (i + 1.0) * (j + 1.0))


def test_matches_numpy_fp64_random():
    A = workloads.uniform((70, 129), seed=7).numpy()
    B = workloads.uniform((129, 45), seed=8).numpy()
    C0 = workloads.uniform((70, 45), seed=9).numpy()
    C, S = oracle.gemm(A, B, alpha=1.5, beta=-2.0, C0=C0)
    ref = 1.5 * (A.astype(np.float64) @ B.astype(np.float64)) - 2.0 * C0
    sref = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64))
    assert np.max(np.abs(C - ref) / (sref + 1.0)) < 1e-13
    assert np.max(np.abs(S - sref) / sref) < 1e-13


def test_entries_closed_form():
    M, N, K = 40, 30, 50
    A, B, Cx = _closed_form_operands(M, N, K)
    rows = np.array([0, 39, 17, 5, 39])
    cols = np.array([0, 29, 3, 28, 0])
    out, s = oracle.gemm_entries(A, B, rows, cols)
    assert np.array_equal(out, Cx[rows, cols])
    assert np.array_equal(s, np.abs(Cx[rows, cols]))
    C0 = np.arange(M * N, dtype=np.float64).reshape(M, N)
    out, _ = oracle.gemm_entries(A, B, rows, cols, alpha=2.0, beta=-1.0, C0=C0)
    assert np.array_equal(out, 2.0 * Cx[rows, cols] - C0[rows, cols])


def test_bf16_inputs_are_exact_in_fp64():
    a, b = workloads.gemm_inputs(33, 17, 65, dtype="bf16", seed=1)
    C, _ = oracle.gemm(a, b)
    ref = a.double().numpy() @ b.double().numpy()
    assert np.max(np.abs(C - ref)) < 1e-12


def test_finite_difference_gradient():
    """L = <G, A B> is linear in every entry of A and B, so a central
    difference in FP64 equals the derivative up to roundoff.  This pins the
    oracle gradient dA = G B^T, dB = A^T G at the (64, 48, 80) shape."""
    M, N, K = workloads.FD_SHAPE
    A = workloads.uniform((M, K), seed=11).numpy().astype(np.float64)
    B = workloads.uniform((K, N), seed=12).numpy().astype(np.float64)
    G = workloads.normal((M, N), seed=13).numpy().astype(np.float64)
    dA, dB = oracle.grad_fp64(A, B, G)

    h = 0.5   # exact perturbation; L is linear so h's size does not matter

    def loss(a, b):
        C, _ = oracle.gemm(a, b, want_abs=False, threads=1)
        return float(np.sum(G * C))

    rng = np.random.default_rng(0)
    ia = rng.choice(M * K, size=96, replace=False)
    for flat in ia:
        i, k = divmod(int(flat), K)
        ap, am = A.copy(), A.copy()
        ap[i, k] += h
        am[i, k] -= h
        fd = (loss(ap, B) - loss(am, B)) / (2 * h)
        scale = np.sum(np.abs(G[i, :]) * np.abs(B[k, :])) + 1.0
        assert abs(fd - dA[i, k]) <= 1e-11 * scale * M * N
    ib = rng.choice(K * N, size=96, replace=False)
    for flat in ib:
        k, j = divmod(int(flat), N)
        bp, bm = B.copy(), B.copy()
        bp[k, j] += h
        bm[k, j] -= h
        fd = (loss(A, bp) - loss(A, bm)) / (2 * h)
        scale = np.sum(np.abs(A[:, k]) * np.abs(G[:, j])) + 1.0
        assert abs(fd - dB[k, j]) <= 1e-11 * scale * M * N


def test_bound_helper():
    S = np.array([[1.0, 2.0]])
    C = np.array([[4.0, -8.0]])
    assert np.allclose(oracle.bound(S, C, "f32"), 5e-5 * S)
    assert np.allclose(oracle.bound(S, C, "bf16"), 5e-5 * S + 2 ** -8 * np.abs(C))


def _table1():
    rows = []
    with open(os.path.join(HERE, "golden", "paper_table1.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            lab, ms, tf, gbs, M, N, K = line.split()
            rows.append((lab, float(ms), float(tf), float(gbs), int(M), int(N), int(K)))
    return rows


def test_paper_table1_accounting():
    """Pin the flop and byte accounting against the paper's Results, Table 1:
    TFLOP/s = 2MNK / t and GB/s = (MK + KN + MN) * 2 B / t reproduce the
    printed columns within their print precision."""
    rows = _table1()
    assert len(rows) == 6
    for lab, ms, tf, gbs, M, N, K in rows:
        flops = workloads.gemm_flops(M, N, K)
        byts = workloads.gemm_bytes(M, N, K, 2, 2, 2)
        t_from_tf = flops / (tf * 1e12) * 1e3          # ms
        # ms is printed to 1e-3 (the rows agree with truncation or rounding)
        assert abs(t_from_tf - ms) <= 0.001, lab
        # the two rate columns share one time, so their ratio is bytes/flops
        assert abs((gbs * 1e9) / (tf * 1e12) - byts / flops) <= 2e-4 * byts / flops, lab


def test_paper_arithmetic_intensity():
    """Methodology: arithmetic intensity 1337 for the 3840x4096x4096 problem
    (2-byte elements).  The accounting gives 1335.6, within 0.2 %."""
    M, N, K = workloads.BF16_SWEEP[0]
    ai = workloads.gemm_flops(M, N, K) / workloads.gemm_bytes(M, N, K, 2, 2, 2)
    assert abs(ai - 1337) / 1337 < 2e-3


def _tf32_trunc(x):
    """x with its low 13 mantissa bits cleared (TF32 by truncation)."""
    return (x.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)


def _tf32_rna(x):
    """x rounded to TF32, nearest with ties away from zero: add half an
    ulp of TF32 to the magnitude bits, then truncate."""
    u = x.view(np.uint32)
    return ((u + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def test_3xtf32_split_meets_the_fp32_bound():
    """The FP32 reading (3xTF32): with x_hi = x truncated to TF32 and
    x_lo = tf32_rn(x - x_hi), a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi.
    Emulated here in numpy (FP32 products of TF32 values are exact; the
    sums run in FP32), the worst error against the FP64 oracle stays
    below 2^-19 of S on mixed-sign and on one-signed inputs, two orders
    under the 5e-5 bound.  One TF32 product alone (the FP32 container
    read truncated, as the MMA reads it) errs by up to 2^-10 per product
    in one direction, and on one-signed inputs the sum's error breaks the
    bound."""
    rng = np.random.default_rng(3)
    M, N, K = 64, 48, 2048
    for lo_v in (-1.0, 0.0):
        a = rng.uniform(lo_v, 1, (M, K)).astype(np.float32)
        b = rng.uniform(lo_v, 1, (K, N)).astype(np.float32)
        ref, S = oracle.gemm(torch.from_numpy(a), torch.from_numpy(b))
        a_hi, b_hi = _tf32_trunc(a), _tf32_trunc(b)
        a_lo, b_lo = _tf32_rna(a - a_hi), _tf32_rna(b - b_hi)
        assert np.all(np.abs(a - a_hi - a_lo) <= np.abs(a) * 2.0 ** -21)   # x_lo carries x - x_hi to 2^-21
        c3 = a_hi @ b_hi + a_hi @ b_lo + a_lo @ b_hi                        # float32 throughout
        rel3 = float((np.abs(c3.astype(np.float64) - ref) / S).max())
        assert rel3 < 2.0 ** -19, (lo_v, rel3)
        if lo_v == 0.0:
            c1 = a_hi @ b_hi
            rel1 = float((np.abs(c1.astype(np.float64) - ref) / S).max())
            assert rel1 > 5e-5, rel1
