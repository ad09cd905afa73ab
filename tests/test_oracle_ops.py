"""Pins of the oracle's reduce, scan, view copy and segmented ops (CPU only):
closed forms, brute force with per-point resolution, invariants between ops,
and NumPy's transpose as a library special case."""
import math
import random

import numpy as np
import pytest

import synth
from oracle import ops as O
from oracle import views as V


def brute_reduce(x, base, ops, out_level):
    """Per-point loop: resolve each logical point on its own."""
    dom = V.domain_shape(base, ops)
    sels = V.selects(base, ops)
    nsel = len(sels)
    nkeep = sum(1 for s in sels if s[0] <= out_level)
    nout = math.prod(dom[:nkeep]) if nkeep else 1
    out = [0] * nout
    flat = np.asarray(x).reshape(-1)
    for p in np.ndindex(*dom):
        e = V.resolve(base, ops, list(p[:nsel]), list(p[nsel:]))
        o = 0
        for c, n in zip(p[:nkeep], dom[:nkeep]):
            o = o * n + c
        out[o] += int(flat[e])
    return O.wrap_i32(out)


def test_closed_forms():
    n = 1000
    x = np.arange(1, n + 1, dtype=np.int32)
    s, _ = O.reduce(x, [n], [], V.GRID)
    assert s[0] == n * (n + 1) // 2
    y, _ = O.scan(x, np.zeros(n, np.int32), [n], [], V.GRID)
    i = np.arange(n, dtype=np.int64)
    assert np.array_equal(y, (i + 1) * (i + 2) // 2)
    ones = np.ones(n, dtype=np.int32)
    y, _ = O.scan(ones, np.zeros(n, np.int32), [n], [], V.GRID)
    assert np.array_equal(y, np.arange(1, n + 1))
    assert O.reduce(ones, [n], [], V.GRID)[0][0] == n


def test_int32_wraps_mod_2_32():
    x = np.array([2**31 - 1, 1, 5], dtype=np.int32)
    assert O.reduce(x, [3], [], V.GRID)[0][0] == -2**31 + 5
    y, _ = O.scan(x, np.zeros(3, np.int32), [3], [], V.GRID)
    assert y.tolist() == [2**31 - 1, -2**31, -2**31 + 5]


def test_fp32_sum_is_exact_on_the_grid():
    x = synth.uniform_grid(1 << 16, seed=3).numpy()
    k = (x.astype(np.float64) * 2**23).astype(np.int64)
    assert np.array_equal(k.astype(np.float64) * 2.0**-23, x.astype(np.float64))
    s, a = O.reduce(x, [x.size], [], V.GRID)
    assert s[0] == k.sum() * 2.0**-23
    assert a[0] == np.abs(k).sum() * 2.0**-23


@pytest.mark.parametrize("seed", range(40))
def test_reduce_brute_force(seed):
    rng = random.Random(seed)
    n = rng.choice([128, 256])
    g = rng.choice([2, 4])
    x = synth.ints_pm1000(n, seed=seed).numpy()
    ops = [("group", n // g, 0), ("select", V.BLOCK, V.X)]
    if rng.random() < 0.5:
        ops.append(("reverse", 0))
    ops += [("group", 32, 0), ("select", V.WARP, V.X), ("select", V.THREAD, V.X)]
    block = (n // g, 1, 1)
    for lvl in (V.GRID, V.BLOCK, V.WARP, V.THREAD):
        want = brute_reduce(x, [n], ops, lvl)
        got, _ = O.reduce(x, [n], ops, lvl, (g, 1, 1), block)
        assert np.array_equal(got, want)


def test_last_scan_element_is_the_reduce():
    for seed in range(5):
        x = synth.ints_pm1000(4096, seed=seed).numpy()
        ops = [("group", 1024, 0), ("select", V.BLOCK, V.X)]
        y, _ = O.scan(x, np.zeros_like(x), [4096], ops, V.BLOCK)
        r, _ = O.reduce(x, [4096], ops, V.BLOCK)
        assert np.array_equal(y.reshape(4, 1024)[:, -1], r)
        # consecutive differences give the input back (integers)
        assert np.array_equal(np.diff(y.reshape(4, 1024).astype(np.int64), axis=1) % 2**32,
                              x.reshape(4, 1024)[:, 1:].astype(np.int64) % 2**32)


def test_scan_through_transpose_is_column_scan():
    x = synth.ints_pm1000(12, seed=1).numpy().reshape(3, 4)
    ops = [("transpose", 0), ("select", V.THREAD, V.X)]
    y, _ = O.scan(x, np.zeros_like(x), [3, 4], ops, V.THREAD, (1, 1, 1), (4, 1, 1))
    want = np.cumsum(x.astype(np.int64), axis=0)
    assert np.array_equal(y, want)


def test_segmented_with_one_segment_is_plain_scan():
    x = synth.uniform_grid(777, seed=2).numpy()
    y, _ = O.scan(x, np.zeros(777), [777], [], V.GRID)
    ys, sums, _, _ = O.segmented_reduce_scan(x, [0, 777])
    assert np.array_equal(ys, y)
    assert sums[0] == O.reduce(x, [777], [], V.GRID)[0][0]


def test_segmented_invariants():
    L = synth.loguniform_lengths(60, seed=4, max_len=300).numpy()
    L[5] = 0
    L[6] = 1
    off = np.concatenate([[0], np.cumsum(L)])
    x = synth.ints_pm1000(int(off[-1]), seed=4).numpy()
    ys, sums, _, _ = O.segmented_reduce_scan(x, off)
    assert sums[5] == 0
    assert ys[off[6]] == x[off[6]]
    for s in range(len(L)):
        if L[s]:
            assert ys[off[s + 1] - 1] == sums[s]
    assert O.wrap_i32(sums.astype(np.int64).sum()) == O.reduce(x, [x.size], [], V.GRID)[0][0]


def test_transpose_matches_numpy_and_involution():
    for R, C in ((33, 65), (1, 17), (17, 1), (64, 64)):
        x = synth.normal_f32(R * C, seed=R).numpy().reshape(R, C)
        t = O.transpose2d(x)
        assert np.array_equal(t, x.T)
        assert np.array_equal(O.transpose2d(t), x)
        via_view = O.view_copy(x, np.zeros((C, R), np.float32), [R, C], [("transpose", 0)], [C, R], [])
        assert np.array_equal(via_view, x.T)


def test_view_copy_leaves_unreached_elements():
    x = np.arange(10, dtype=np.float32)
    out = O.view_copy(x, np.full(10, -7.0, np.float32), [10], [("split_fst", 4, 0)], [10], [("split_snd", 6, 0)])
    assert out.tolist() == [-7.0] * 6 + [0.0, 1.0, 2.0, 3.0]


# ---- other operators: maximum, minimum, exclusive scans ----------------------
def test_max_min_closed_forms():
    n = 1000
    x = np.arange(1, n + 1, dtype=np.int32)[::-1].copy()            # n .. 1
    assert O.reduce_op(x, [n], [], V.GRID, "max")[0] == n
    assert O.reduce_op(x, [n], [], V.GRID, "min")[0] == 1
    # per block of 10: the block's first element is its maximum (decreasing data)
    got = O.reduce_op(x, [n], [("group", 10, 0), ("select", V.BLOCK, V.X)], V.BLOCK, "max")
    assert np.array_equal(got, x[::10])
    xf = np.array([-3.5, -1.25, -7.0], np.float32)
    assert O.reduce_op(xf, [3], [], V.GRID, "max")[0] == -1.25   # all negative: not 0
    assert O.reduce_op(xf, [3], [], V.GRID, "min")[0] == -7.0


def test_max_ignores_nan_and_identity_of_empty():
    xf = np.array([np.nan, 2.0, np.nan, -1.0], np.float32)
    assert O.reduce_op(xf, [4], [], V.GRID, "max")[0] == 2.0
    assert O.reduce_op(xf, [4], [], V.GRID, "min")[0] == -1.0
    assert np.isnan(O.reduce_op(np.array([np.nan], np.float32), [1], [], V.GRID, "max")[0])
    _, tot, _, _ = O.segmented_op(np.zeros(3, np.int32), [0, 0, 3], "max")
    assert tot[0] == np.iinfo(np.int32).min and tot[1] == 0
    _, tot, _, _ = O.segmented_op(np.zeros(3, np.float32), [0, 3, 3], "min")
    assert tot[1] == np.inf


def test_exclusive_scan_closed_forms():
    n = 500
    ones = np.ones(n, np.int32)
    out, _ = O.scan_op(ones, np.zeros(n, np.int32), [n], [], V.GRID, "sum", True)
    assert np.array_equal(out, np.arange(n))                          # i ones before point i
    x = np.arange(1, n + 1, dtype=np.int32)
    out, _ = O.scan_op(x, np.zeros(n, np.int32), [n], [], V.GRID, "sum", True)
    i = np.arange(n)
    assert np.array_equal(out, i * (i + 1) // 2)
    out, _ = O.scan_op(x, np.zeros(n, np.int32), [n], [], V.GRID, "max", True)
    assert out[0] == np.iinfo(np.int32).min and np.array_equal(out[1:], x[:-1])   # increasing data
    out, _ = O.scan_op(x, np.zeros(n, np.int32), [n], [], V.GRID, "min", False)
    assert np.all(out == 1)


def test_operators_brute_force_small():
    rng = np.random.default_rng(7)
    for trial in range(20):
        m = int(rng.integers(1, 9))
        g = int(rng.integers(1, 9))
        n = m * g
        x = rng.integers(-50, 50, size=n).astype(np.int32)
        ops = [("group", m, 0), ("select", V.BLOCK, V.X)]
        for op, f in (("max", max), ("min", min)):
            want = [f(x[k * m:(k + 1) * m].tolist()) for k in range(g)]
            assert O.reduce_op(x, [n], ops, V.BLOCK, op).tolist() == want
            for excl in (False, True):
                got, _ = O.scan_op(x, np.zeros(n, np.int32), [n], ops, V.BLOCK, op, excl)
                for k in range(g):
                    seg = x[k * m:(k + 1) * m].tolist()
                    for i in range(m):
                        part = seg[:i] if excl else seg[:i + 1]
                        exp = f(part) if part else (-2 ** 31 if op == "max" else 2 ** 31 - 1)
                        assert got[k * m + i] == exp
        # exclusive sums are the inclusive ones shifted within each segment
        inc, _ = O.scan_op(x, np.zeros(n, np.int32), [n], ops, V.BLOCK, "sum", False)
        exc, _ = O.scan_op(x, np.zeros(n, np.int32), [n], ops, V.BLOCK, "sum", True)
        assert np.array_equal(inc - x, exc)


def test_segmented_operators_match_per_segment_definition():
    rng = np.random.default_rng(11)
    L = rng.integers(0, 7, size=30)
    off = np.concatenate([[0], np.cumsum(L)])
    x = rng.integers(-9, 9, size=int(off[-1])).astype(np.int32)
    for op in ("sum", "max", "min"):
        for excl in (False, True):
            sc, tot, _, _ = O.segmented_op(x, off, op, excl)
            for s in range(30):
                a, b = off[s], off[s + 1]
                want, _ = O.scan_op(x[a:b], np.zeros(b - a, np.int32), [int(b - a)], [], V.GRID, op, excl) \
                    if b > a else (np.zeros(0, np.int32), None)
                assert np.array_equal(sc[a:b], want)
                if b > a and not excl:
                    assert tot[s] == sc[b - 1]          # total = last inclusive value


# ---- pins of the caller-chosen operators (product, bitwise, arg-max / arg-min)
def test_int_product_closed_forms():
    # powers of two: 2^(sum k) modulo 2^32
    ks = [3, 5, 7, 11, 2, 1]
    x = np.array([1 << k for k in ks], np.int32)
    got = O.reduce_op(x, [6], [], V.GRID, "prod")[0]
    assert int(got) == (1 << 29)
    assert int(O.reduce_op(np.array([65536, 65536], np.int32), [2], [], V.GRID, "prod")[0]) == 0
    assert int(O.reduce_op(np.full(7, -1, np.int32), [7], [], V.GRID, "prod")[0]) == -1
    # 3^20 modulo 2^32 through Python's modular pow, as a signed int32
    p = pow(3, 20, 1 << 32)
    assert int(O.reduce_op(np.full(20, 3, np.int32), [20], [], V.GRID, "prod")[0]) == (p - (1 << 32) if p >= 1 << 31 else p)
    # the scan's prefixes are the powers
    sc, _ = O.scan_op(np.full(20, 3, np.int32), np.zeros(20, np.int32), [20], [], V.GRID, "prod")
    want = [pow(3, i + 1, 1 << 32) for i in range(20)]
    assert [int(v) & 0xFFFFFFFF for v in sc] == want


def test_float_product_against_exact_fractions():
    from fractions import Fraction
    rng = np.random.default_rng(5)
    x = (1.0 + rng.uniform(-1, 1, 300) * 2.0 ** -6).astype(np.float32)
    exact = Fraction(1)
    for v in x.tolist():
        exact *= Fraction(v)
    got = O.reduce_op(x, [300], [], V.GRID, "prod")[0]
    assert abs(Fraction(float(got)) - exact) <= Fraction(299, 1 << 53) * abs(exact) * 2
    assert O.reduce_op(np.array([2, 0.5, 4, 0.25], np.float32), [4], [], V.GRID, "prod")[0] == 1.0
    u = 2.0 ** -24
    assert O.prod_tolerance(1) == 0.0 and abs(O.prod_tolerance(3) - 2 * u) <= 8 * u * u


def test_bitwise_closed_forms_and_brute_force():
    import functools
    import operator
    xs = np.arange(64, dtype=np.int32)                   # xor of 0 .. 4k - 1 is 0
    assert int(O.reduce_op(xs, [64], [], V.GRID, "xor")[0]) == 0
    pw = np.array([1 << k for k in (0, 3, 9, 30)], np.int32)
    assert int(O.reduce_op(pw, [4], [], V.GRID, "or")[0]) == int(pw.astype(np.int64).sum())
    assert int(O.reduce_op(np.array([0x5A5A5A5A, ~0x5A5A5A5A], np.int32), [2], [], V.GRID, "and")[0]) == 0
    rng = np.random.default_rng(7)
    x = rng.integers(-2 ** 31, 2 ** 31, 50).astype(np.int32)
    for op, f in (("and", operator.and_), ("or", operator.or_), ("xor", operator.xor)):
        sc, _ = O.scan_op(x, np.zeros(50, np.int32), [50], [], V.GRID, op)
        for p in range(50):
            assert int(sc[p]) == functools.reduce(f, [int(v) for v in x[:p + 1]])
        ex, _ = O.scan_op(x, np.zeros(50, np.int32), [50], [], V.GRID, op, True)
        assert int(ex[0]) == O.identity(op, True) and np.array_equal(ex[1:], sc[:-1])


def _brute_arg(vals, idx, op):
    """Brute force: among the non-NaN values the best, then the smallest
    index (all NaN: the smallest index)."""
    pairs = [(float(v), int(i)) for v, i in zip(vals, idx)]
    if not pairs:
        return -1
    num = [p for p in pairs if not math.isnan(p[0])] or [(0.0, p[1]) for p in pairs]
    if op == "argmax":
        return max(num, key=lambda p: (p[0], -p[1]))[1]
    return min(num, key=lambda p: (p[0], p[1]))[1]


def test_arg_operators_brute_force():
    rng = np.random.default_rng(9)
    for trial in range(40):
        n = int(rng.integers(1, 40))
        x = rng.integers(-3, 4, n).astype(np.float32)    # many ties
        if trial % 3 == 0:
            x[rng.integers(0, n, 3)] = np.nan
        if trial % 5 == 0:
            x[:] = np.nan
        for op in ("argmax", "argmin"):
            assert int(O.reduce_op(x, [n], [], V.GRID, op)[0]) == _brute_arg(x, range(n), op)
            # through a reversed view the indices stay base-array indices
            assert int(O.reduce_op(x, [n], [("reverse", 0)], V.GRID, op)[0]) == _brute_arg(x, range(n), op)
            sc, _ = O.scan_op(x, np.zeros(n, np.int32), [n], [], V.GRID, op)
            rv, _ = O.scan_op(x, np.zeros(n, np.int32), [n], [("reverse", 0)], V.GRID, op)
            for p in range(n):
                assert int(sc[p]) == _brute_arg(x[:p + 1], range(p + 1), op)
                # reversed: point p of the view is element n-1-p; its prefix is elements n-1-p .. n-1
                assert int(rv[n - 1 - p]) == _brute_arg(x[n - 1 - p:], range(n - 1 - p, n), op)
            ex, _ = O.scan_op(x, np.zeros(n, np.int32), [n], [], V.GRID, op, True)
            assert int(ex[0]) == -1 and np.array_equal(ex[1:], sc[:-1])
    xi = np.array([4, 9, 9, -2, 9], np.int32)
    assert int(O.reduce_op(xi, [5], [], V.GRID, "argmax")[0]) == 1
    assert int(O.reduce_op(xi, [5], [], V.GRID, "argmin")[0]) == 3
    assert int(O.reduce_op(np.array([0.0, -0.0], np.float32), [2], [], V.GRID, "argmin")[0]) == 0


def test_new_operators_segmented_match_scans():
    rng = np.random.default_rng(13)
    L = rng.integers(0, 9, size=25)
    off = np.concatenate([[0], np.cumsum(L)])
    x = rng.integers(-4, 5, size=int(off[-1])).astype(np.int32)
    for op in ("prod", "and", "or", "xor", "argmax", "argmin"):
        for excl in (False, True):
            sc, tot, _, _ = O.segmented_op(x, off, op, excl)
            for s in range(25):
                a, b = int(off[s]), int(off[s + 1])
                if b == a:
                    assert int(tot[s]) == O.identity(op, True)
                    continue
                want, _ = O.scan_op(x[a:b], np.zeros(b - a, np.int32), [b - a], [], V.GRID, op, excl)
                if op.startswith("arg"):
                    want = np.where(want >= 0, want + a, want)   # indices into the whole array
                    assert int(tot[s]) == _brute_arg(x[a:b], range(a, b), op)
                assert np.array_equal(sc[a:b], want)
