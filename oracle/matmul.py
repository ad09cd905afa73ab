"""Oracle: matrix multiplication and the BF16 split (test infrastructure).

Section 5 lists matrix multiplication among its benchmarks without fixing the
data type.  Reading: C = A B with FP32 row-major A (M x K), B (K x N) and FP32
C; the reference value is the FP64 product of the exactly widened inputs.

Split precision: every FP32 value a is written as a0 + a1 + a2 with
  a0 = bf16(a), a1 = bf16(a - a0), a2 = bf16(a - a0 - a1)
where bf16() rounds to the nearest BF16 number, ties to even, and the
subtractions are FP32 (exact, because each a_i holds the leading bits of what
is left).  The product keeps the six partial products A_i B_j with i + j <= 2.
"""
from __future__ import annotations

import numpy as np


def matmul_f64(A, B):
    """Reference product in FP64 (library GEMM on widened inputs)."""
    return np.asarray(A, dtype=np.float64) @ np.asarray(B, dtype=np.float64)


def matmul_rows_f64(A, B, rows):
    """Reference product restricted to some rows of C."""
    return np.asarray(A, dtype=np.float64)[rows] @ np.asarray(B, dtype=np.float64)


def matmul_naive(A, B):
    """Triple loop, for tiny shapes only: C[i][j] = sum_k A[i][k] B[k][j]."""
    M, K = len(A), len(A[0])
    N = len(B[0])
    C = [[0.0] * N for _ in range(M)]
    for i in range(M):
        for j in range(N):
            s = 0.0
            for k in range(K):
                s += float(A[i][k]) * float(B[k][j])
            C[i][j] = s
    return np.array(C)


def bf16_rne(x):
    """FP32 -> nearest BF16 (ties to even), returned as FP32 values.

    On the bit pattern: add 0x7FFF plus the lowest kept bit, then clear the 16
    low bits.  A carry out of the mantissa bumps the exponent, which is the
    correct rounding (including overflow to infinity).  NaNs stay NaN (quiet).
    """
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = x.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = ((b + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    nan = np.isnan(x)
    r[nan] = (b[nan].astype(np.uint32) | np.uint32(0x00400000)) & np.uint32(0xFFFF0000)
    return r.view(np.float32)


def split3(a):
    """(a0, a1, a2), each holding BF16 values (stored as FP32)."""
    a = np.asarray(a, dtype=np.float32)
    a0 = bf16_rne(a)
    r1 = (a - a0).astype(np.float32)
    a1 = bf16_rne(r1)
    r2 = (r1 - a1).astype(np.float32)
    a2 = bf16_rne(r2)
    return a0, a1, a2


def split3_product_f64(A, B):
    """sum_{i+j<=2} A_i B_j in FP64: the value the split method approximates,
    separating its representation error from accumulation error."""
    As, Bs = split3(A), split3(B)
    C = np.zeros((np.shape(A)[0], np.shape(B)[1]), dtype=np.float64)
    for i in range(3):
        for j in range(3 - i):
            C += As[i].astype(np.float64) @ Bs[j].astype(np.float64)
    return C


def rel_frobenius(C, C_ref):
    """||C - C_ref||_F / ||C_ref||_F in FP64."""
    C = np.asarray(C, dtype=np.float64)
    C_ref = np.asarray(C_ref, dtype=np.float64)
    return float(np.linalg.norm(C - C_ref) / np.linalg.norm(C_ref))
