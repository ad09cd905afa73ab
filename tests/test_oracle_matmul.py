"""Pins of the oracle's matmul, BF16 rounding and split (CPU only)."""
import json
import os

import numpy as np

import synth
from oracle import matmul as M

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_f64_product_vs_triple_loop():
    A = synth.normal_f32(5 * 7, seed=1).numpy().reshape(5, 7)
    B = synth.normal_f32(7 * 3, seed=2).numpy().reshape(7, 3)
    assert np.allclose(M.matmul_f64(A, B), M.matmul_naive(A, B), rtol=0, atol=1e-12)
    rows = [0, 3]
    assert np.array_equal(M.matmul_rows_f64(A, B, rows), M.matmul_f64(A, B)[rows])


def test_closed_forms():
    B = synth.normal_f32(16 * 9, seed=3).numpy().reshape(16, 9)
    assert np.array_equal(M.matmul_f64(np.eye(16, dtype=np.float32), B), B.astype(np.float64))
    K = 37
    assert np.array_equal(M.matmul_f64(np.ones((4, K), np.float32), np.ones((K, 6), np.float32)),
                          np.full((4, 6), float(K)))
    u = synth.normal_f32(8, seed=4).numpy()
    v = synth.normal_f32(5, seed=5).numpy()
    A = np.repeat(u[:, None], K, axis=1)          # rows constant
    Bm = np.repeat(v[None, :], K, axis=0)         # columns constant
    C = M.matmul_f64(A, Bm)
    assert np.allclose(C, K * np.outer(u.astype(np.float64), v.astype(np.float64)), rtol=1e-14, atol=0)


def test_bf16_golden_values():
    g = json.load(open(os.path.join(GOLD, "bf16_rne.json")))
    for src, want, why in g["cases"]:
        x = np.array([int(src, 16)], dtype=np.uint32).view(np.float32)
        got = M.bf16_rne(x).view(np.uint32)[0]
        assert got == int(want, 16), why
    nan = np.array([0x7fc00001], dtype=np.uint32).view(np.float32)
    assert np.isnan(M.bf16_rne(nan))[0]


def test_bf16_against_neighbour_search():
    """Independent route: take the two BF16 numbers around x and pick the
    nearer in FP64, the one with an even last bit on a tie."""
    bits = (synth.splitmix64(synth.stream_key(9), 0, 20000) & 0xFFFFFFFF).numpy().astype(np.uint32)
    x = bits.view(np.float32)
    ok = np.isfinite(x) & (np.abs(x) < 3.3e38)
    x = x[ok]
    got = M.bf16_rne(x)
    b = x.view(np.uint32)
    lo = (b & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)
    hi = ((b & np.uint32(0xFFFF0000)) + np.uint32(0x10000)).view(np.float32).astype(np.float64)
    xd = x.astype(np.float64)
    dlo, dhi = np.abs(xd - lo), np.abs(hi - xd)
    lo_even = ((b >> np.uint32(16)) & np.uint32(1)) == 0
    pick_lo = (dlo < dhi) | ((dlo == dhi) & lo_even)
    want = np.where(pick_lo, lo, hi)
    assert np.array_equal(got.astype(np.float64), want)


def test_split3_reconstructs():
    a = synth.normal_f32(1 << 16, seed=6).numpy()
    a0, a1, a2 = M.split3(a)
    for t in (a0, a1, a2):
        assert np.array_equal(M.bf16_rne(t), t)          # each term is a BF16 number
    err = np.abs(a.astype(np.float64) - (a0.astype(np.float64) + a1 + a2))
    assert np.all(err <= 2.0**-24 * np.abs(a.astype(np.float64)))
    assert np.mean(err == 0) > 0.99
    # term magnitudes fall by at least 2^-8 each
    nz = a1 != 0
    assert np.all(np.abs(a1[nz]) <= 2.0**-8 * np.abs(a0[nz]))


def test_split_product_close_to_f64():
    A = synth.normal_f32(64 * 96, seed=7).numpy().reshape(64, 96)
    B = synth.normal_f32(96 * 48, seed=8).numpy().reshape(96, 48)
    e = M.rel_frobenius(M.split3_product_f64(A, B), M.matmul_f64(A, B))
    assert e < 1e-6
    # a single BF16 term is much coarser (unit roundoff 2^-9 per factor)
    e1 = M.rel_frobenius(M.matmul_f64(M.bf16_rne(A), M.bf16_rne(B)), M.matmul_f64(A, B))
    assert 1e-4 < e1 < 1e-2


def test_rel_frobenius():
    assert M.rel_frobenius([[3.0, 4.0]], [[3.0, 4.0]]) == 0.0
    assert abs(M.rel_frobenius([[3.0, 5.0]], [[3.0, 4.0]]) - 0.2) < 1e-15
