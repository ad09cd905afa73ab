"""Caller-chosen associative operators on the GPU against the oracle: product
(int32 modulo 2^32, FP32 within gamma_(m-1)), bitwise and / or / xor (int32)
and arg-maximum / arg-minimum (int32 element indices of the base array,
ties to the smallest index), for reduce (plain, per-level outputs, general
maps), scan (plain, per-level segments, general views in one pass,
exclusive, in place) and the CSR-segmented call.  Integer results and
indices are compared bit for bit; FP32 products within the bound of
oracle.ops.prod_tolerance."""
import numpy as np
import pytest
import torch

import paper_2305_03448_gb300 as D
import synth
from oracle import ops as O
from oracle import views as V

pytestmark = pytest.mark.gpu
FLAG = {"prod": D.PROD, "and": D.AND, "or": D.OR, "xor": D.XOR, "argmax": D.ARGMAX, "argmin": D.ARGMIN,
        "sum": 0, "max": D.MAX, "min": D.MIN}
INT_OPS = ["prod", "and", "or", "xor", "argmax", "argmin"]
FLOAT_OPS = ["prod", "argmax", "argmin"]


@pytest.fixture(scope="module", autouse=True)
def _lib(desc_lib):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return desc_lib


def data(op, dtype, n, seed):
    """Inputs that keep each operator's results informative: odd factors
    for int32 products (never 0 modulo 2^32), factors near 1 for FP32
    products, scrambled 32-bit patterns for the bitwise operators, and
    values with many ties for the arg operators."""
    if dtype == "i32":
        x = synth.ints_pm1000(n, seed=seed)
        if op == "prod":
            return (x % 4) * 2 + 1 - 8 * (x < 0).to(torch.int32)
        if op in ("and", "or", "xor"):
            return (x.to(torch.int64) * 2654435761 + 12345).to(torch.int32)
        return x
    x = synth.uniform_grid(n, seed=seed)
    if op == "prod":
        return 1.0 + x * (2.0 ** -7)
    return x


def check_values(got, want, op, is_int, m):
    got = np.asarray(got)
    if is_int or op.startswith("arg"):
        assert np.array_equal(got.astype(np.int64), np.asarray(want).astype(np.int64))
    elif op in ("max", "min"):
        assert np.array_equal(got.astype(np.float64), np.asarray(want, dtype=np.float64))
    else:
        want = np.asarray(want, dtype=np.float64)
        assert np.all(np.abs(got.astype(np.float64) - want) <= O.prod_tolerance(m) * np.abs(want) + 1e-37)


@pytest.mark.parametrize("n", [1, 77, 4097, (1 << 20) + 5, 3_000_001])
@pytest.mark.parametrize("dtype,op", [("i32", o) for o in INT_OPS] + [("f32", o) for o in FLOAT_OPS])
def test_reduce(n, dtype, op):
    x = data(op, dtype, n, n + 1)
    got = D.desc_reduce(x.cuda(), [n], [], V.GRID, flags=FLAG[op]).cpu().numpy()
    check_values(got, O.reduce_op(x.numpy(), [n], [], V.GRID, op), op, dtype == "i32", n)


@pytest.mark.parametrize("dtype,op", [("i32", o) for o in INT_OPS] + [("f32", o) for o in FLOAT_OPS])
def test_reduce_views(dtype, op):
    n = 1 << 18
    x = data(op, dtype, n, 3)
    views = [([("group", 1024, 0), ("select", V.BLOCK, V.X), ("group", 32, 0), ("select", V.WARP, V.X),
               ("select", V.THREAD, V.X)], V.BLOCK, (n // 1024, 1, 1), (1024, 1, 1), 1024),
             ([("group", 16, 0), ("select", V.BLOCK, V.X)], V.BLOCK, (n // 16, 1, 1), (1, 1, 1), 16),
             ([("group", 512, 0), ("select", V.BLOCK, V.X)], V.BLOCK, (n // 512, 1, 1), (1, 1, 1), 512),
             ([("reverse", 0), ("group", 8192, 0), ("select", V.BLOCK, V.X)], V.BLOCK, (n // 8192, 1, 1),
              (1, 1, 1), 8192),
             ([("group", 64, 0), ("reverse", 0), ("transpose", 0), ("select", V.BLOCK, V.X)], V.BLOCK, (64, 1, 1),
              (1, 1, 1), n // 64)]
    for ops, lvl, g, b, m in views:
        got = D.desc_reduce(x.cuda(), [n], ops, lvl, g, b, flags=FLAG[op]).cpu().numpy()
        check_values(got, O.reduce_op(x.numpy(), [n], ops, lvl, op, g, b), op, dtype == "i32", m)
    D.desc_force_generic(True)
    try:
        ops, lvl, g, b, m = views[0]
        got = D.desc_reduce(x.cuda(), [n], ops, lvl, g, b, flags=FLAG[op]).cpu().numpy()
        check_values(got, O.reduce_op(x.numpy(), [n], ops, lvl, op, g, b), op, dtype == "i32", m)
    finally:
        D.desc_force_generic(False)


@pytest.mark.parametrize("op", INT_OPS)
def test_reduce_empty_gives_the_identity(op):
    out = D.desc_reduce(torch.zeros(8, dtype=torch.int32).cuda(), [8], [("split_fst", 0, 0)], V.GRID,
                        flags=FLAG[op])
    assert int(out.item()) == O.identity(op, True)


def test_flags_are_checked():
    x = torch.zeros(64).cuda()
    for flags in (D.AND, D.OR, D.XOR, D.PROD | D.MAX, D.ARGMAX | D.ARGMIN, D.KAHAN | D.PROD):
        with pytest.raises(D.DescError) as e:
            D.desc_reduce(x, [64], [], V.GRID, flags=flags)
        assert e.value.status == 1
    with pytest.raises(D.DescError):
        D.desc_scan(x, [64], [], V.GRID, flags=D.XOR)
    with pytest.raises(D.DescError):
        D.desc_scan(torch.zeros(64, dtype=torch.int32).cuda(), [64], [], V.GRID, flags=D.KAHAN)


def check_scan(x, op, excl, ops=(), lvl=V.GRID, g=None, b=None, inplace=False, seg_len=None):
    n = x.numel()
    flags = FLAG[op] | (D.EXCLUSIVE if excl else 0)
    xd = x.cuda()
    arg = op.startswith("arg")
    if inplace:
        out = xd
    else:
        out = torch.zeros(n, dtype=torch.int32 if arg else x.dtype, device="cuda")
    init = (x.numpy() if not arg else x.numpy().view(np.int32)) if inplace else np.zeros(
        n, np.int32 if arg else x.numpy().dtype)
    got = D.desc_scan(xd, [n], list(ops), lvl, g, b, out=out, flags=flags).cpu().numpy()
    if arg and inplace:
        got = got.view(np.int32)
    want, _ = O.scan_op(x.numpy(), init, [n], list(ops), lvl, op, excl, g, b)
    check_values(got, want, op, x.dtype == torch.int32, seg_len or n)


@pytest.mark.parametrize("n", [1, 5, 4096, 4097, 16385, 3 * 4096 + 11, 200_003])
@pytest.mark.parametrize("op", INT_OPS)
@pytest.mark.parametrize("excl", [False, True])
def test_scan_int(n, op, excl):
    check_scan(data(op, "i32", n, n), op, excl)


@pytest.mark.parametrize("n", [1, 4097, 200_003])
@pytest.mark.parametrize("op", FLOAT_OPS)
@pytest.mark.parametrize("excl", [False, True])
def test_scan_float(n, op, excl):
    check_scan(data(op, "f32", n, n + 7), op, excl)


@pytest.mark.parametrize("m", [7, 4096, 5000, 70000])
@pytest.mark.parametrize("op", ["prod", "xor", "argmax", "argmin"])
def test_scan_segments_per_block(m, op):
    g = max(1, 300000 // m)
    for dtype in ("i32", "f32") if op in FLOAT_OPS else ("i32",):
        x = data(op, dtype, g * m, m)
        check_scan(x, op, m % 2 == 0, [("group", m, 0), ("select", V.BLOCK, V.X)], V.BLOCK, (g, 1, 1), (1, 1, 1),
                   seg_len=m)


@pytest.mark.parametrize("op", INT_OPS + ["sum", "max", "min"])
def test_scan_general_views_one_pass(op):
    """Views whose lowered map is not one contiguous run: the scan gathers
    through the map in its loads and scatters in its stores."""
    n = 3 * 64 * 257
    x = data(op, "i32", n, 41) if op in INT_OPS else synth.ints_pm1000(n, seed=41)
    cases = [([("reverse", 0)], V.GRID, None, None),
             ([("group", 257, 0), ("transpose", 0)], V.GRID, None, None),                # columns of [192][257]
             ([("group", 257, 0), ("transpose", 0), ("select", V.BLOCK, V.X)], V.BLOCK, (257, 1, 1), (1, 1, 1)),
             ([("group", 64, 0), ("reverse", 1)], V.GRID, None, None),                    # map(reverse)
             ([("split_snd", 1001, 0), ("reverse", 0)], V.GRID, None, None),
             ([("group", 257, 0), ("group", 8, 0), ("transpose", 0)], V.GRID, None, None)]   # three map dims
    for ops, lvl, g, b in cases:
        for excl in (False, True):
            check_scan(x, op, excl, ops, lvl, g, b)
    check_scan(x, op, False, cases[0][0], inplace=True)
    if op in FLOAT_OPS or op in ("sum", "max", "min"):
        xf = data(op, "f32", n, 42) if op in FLOAT_OPS else synth.uniform_grid(n, seed=42)
        for ops, lvl, g, b in cases[:3]:
            if op == "sum":
                flags = 0
                got = D.desc_scan(xf.cuda(), [n], ops, lvl, g, b, flags=flags).cpu().numpy()
                want, pa = O.scan_op(xf.numpy(), np.zeros(n, np.float32), [n], ops, lvl, "sum", False, g, b)
                assert np.all(np.abs(got - want) <= 1e-5 * pa + 1e-30)
            else:
                check_scan(xf, op, False, ops, lvl, g, b)


@pytest.mark.parametrize("op", INT_OPS)
@pytest.mark.parametrize("excl", [False, True])
def test_segmented_csr(op, excl):
    L = synth.loguniform_lengths(700, seed=17, max_len=30000)
    L[::9] = 0
    off = synth.offsets_from_lengths(L)
    flags = FLAG[op] | (D.EXCLUSIVE if excl else 0)
    dtypes = ("i32", "f32") if op in FLOAT_OPS else ("i32",)
    for dtype in dtypes:
        x = data(op, dtype, int(off[-1]), 19)
        sc, tot = D.desc_segmented_reduce_scan(x.cuda(), off.cuda(), flags=flags)
        want, wtot, _, _ = O.segmented_op(x.numpy(), off.numpy(), op, excl)
        m = int(L.max())
        check_values(sc.cpu().numpy(), want, op, dtype == "i32", m)
        check_values(tot.cpu().numpy(), wtot, op, dtype == "i32", m)
    # every segment empty: the totals are the identity
    off0 = torch.zeros(4, dtype=torch.int64)
    _, tot = D.desc_segmented_reduce_scan(torch.zeros(0, dtype=torch.int32).cuda(), off0.cuda(), flags=flags)
    assert np.array_equal(tot.cpu().numpy(), np.full(3, O.identity(op, True), np.int32))


def test_arg_nan_ties_and_signed_zero():
    x = torch.tensor([float("nan"), 2.0, -0.0, 2.0, 0.0, float("nan"), -7.0])
    assert D.desc_reduce(x.cuda(), [7], [], V.GRID, flags=D.ARGMAX).item() == 1
    assert D.desc_reduce(x.cuda(), [7], [], V.GRID, flags=D.ARGMIN).item() == 6
    z = torch.tensor([0.0, -0.0, 0.0])
    assert D.desc_reduce(z.cuda(), [3], [("reverse", 0)], V.GRID, flags=D.ARGMIN).item() == 0
    allnan = torch.full((5,), float("nan"))
    assert D.desc_reduce(allnan.cuda(), [5], [("reverse", 0)], V.GRID, flags=D.ARGMAX).item() == 0
    got = D.desc_scan(x.cuda(), [7], [], V.GRID, flags=D.ARGMAX).cpu().numpy()
    want, _ = O.scan_op(x.numpy(), np.zeros(7, np.int32), [7], [], V.GRID, "argmax")
    assert np.array_equal(got, want)
    # ties across tiles and CTAs: a constant array picks element 0 (scan: each prefix picks 0)
    n = 1_000_003
    c = torch.full((n,), 5, dtype=torch.int32)
    assert D.desc_reduce(c.cuda(), [n], [], V.GRID, flags=D.ARGMAX).item() == 0
    assert D.desc_reduce(c.cuda(), [n], [("reverse", 0)], V.GRID, flags=D.ARGMIN).item() == 0
    s = D.desc_scan(c.cuda(), [n], [("reverse", 0)], V.GRID, flags=D.ARGMAX).cpu().numpy()
    assert np.array_equal(s, np.arange(n, dtype=np.int32))   # prefix of the reversed view ends at element i


def test_large_sampled():
    """2^26 points: the arg-maximum scan at sampled positions, each checked
    against the oracle's arg_pick over its prefix; the odd-factor product."""
    n = 1 << 26
    x = synth.ints_pm1000(n, seed=23)
    got = D.desc_scan(x.cuda(), [n], [], V.GRID, flags=D.ARGMAX).cpu().numpy()
    xn = x.numpy()
    rng = np.random.default_rng(1)
    for p in list(rng.integers(0, n, 6)) + [n - 1, 0, 4095, 4096]:
        assert int(got[p]) == O.arg_pick(xn[:p + 1], np.arange(p + 1), "argmax")
    xp = data("prod", "i32", n, 29)
    got = D.desc_reduce(xp.cuda(), [n], [], V.GRID, flags=D.PROD).item()
    # the product modulo 2^32 from the value counts (Python's modular pow)
    acc = 1
    vals, cnt = np.unique(xp.numpy(), return_counts=True)
    for v, c in zip(vals.tolist(), cnt.tolist()):
        acc = (acc * pow(int(v) & 0xFFFFFFFF, int(c), 1 << 32)) & 0xFFFFFFFF
    assert (int(got) & 0xFFFFFFFF) == acc


@pytest.mark.parametrize("n", [5, 8191, 3 * 8192 + 5, 200_003])
def test_arg_scan_closed_forms(n):
    """Monotone inputs, where every point beats (or never beats) its prefix:
    the running arg-maximum of an increasing array is p and its arg-minimum 0;
    of a decreasing array the reverse.  Arrays of INT_MIN or INT_MAX (order
    code 0 under arg-maximum or arg-minimum) keep element 0 throughout; the
    exclusive form is -1 at 0 and the inclusive value shifted by one."""
    p = np.arange(n, dtype=np.int64)
    up = torch.arange(n, dtype=torch.int32)
    down = torch.flip(up, [0]).contiguous()
    upf = up.to(torch.float32) - n / 2.0                     # exact in FP32 for these n
    cases = [(up, D.ARGMAX, p), (up, D.ARGMIN, 0 * p), (down, D.ARGMAX, 0 * p), (down, D.ARGMIN, p),
             (upf, D.ARGMAX, p), (-upf, D.ARGMIN, p)]
    for v in (-2 ** 31, 2 ** 31 - 1):
        c = torch.full((n,), v, dtype=torch.int32)
        cases += [(c, D.ARGMAX, 0 * p), (c, D.ARGMIN, 0 * p)]
    for x, flags, want in cases:
        got = D.desc_scan(x.cuda(), [n], [], V.GRID, flags=flags).cpu().numpy()
        assert np.array_equal(got.astype(np.int64), want), (x[:3], flags)
        ex = D.desc_scan(x.cuda(), [n], [], V.GRID, flags=flags | D.EXCLUSIVE).cpu().numpy()
        assert ex[0] == -1 and np.array_equal(ex[1:].astype(np.int64), want[:-1])


@pytest.mark.parametrize("op", ["argmax", "argmin"])
def test_arg_scan_unaligned_buffers(op):
    """Input and output that start 4 bytes past a 16-byte boundary take the
    scan's single-element loads and stores; the result is the oracle's."""
    n = 3 * 8192 + 7
    for dtype in ("i32", "f32"):
        x = data(op, dtype, n + 1, 31)
        xd = x.cuda()[1:]
        out = torch.zeros(n + 1, dtype=torch.int32, device="cuda")[1:]
        assert xd.data_ptr() % 16 and out.data_ptr() % 16
        for excl in (False, True):
            flags = FLAG[op] | (D.EXCLUSIVE if excl else 0)
            got = D.desc_scan(xd, [n], [], V.GRID, out=out, flags=flags).cpu().numpy()
            want, _ = O.scan_op(x[1:].numpy(), np.zeros(n, np.int32), [n], [], V.GRID, op, excl)
            assert np.array_equal(got.astype(np.int64), np.asarray(want).astype(np.int64))


@pytest.mark.parametrize("op", ["argmax", "argmin"])
def test_arg_scan_mapped_many_tiles(op):
    """Arg scans through maps of one and two dims over many 8192-point tiles,
    with many ties (ties go to the smallest base index, which a reversed or
    column view visits last): a reversed array, the columns of a matrix as
    one scan and as one segment per column, every view inclusive and
    exclusive, int32 and FP32, against the oracle."""
    R, C = 301, 997
    n = R * C
    cases = [([("reverse", 0)], V.GRID, None, None),
             ([("group", C, 0), ("transpose", 0)], V.GRID, None, None),
             ([("group", C, 0), ("transpose", 0), ("select", V.BLOCK, V.X)], V.BLOCK, (C, 1, 1), (1, 1, 1)),
             ([("group", C, 0), ("reverse", 1), ("select", V.BLOCK, V.X)], V.BLOCK, (R, 1, 1), (1, 1, 1))]
    for dtype in ("i32", "f32"):
        x = data(op, dtype, n, 53)
        for ops, lvl, g, b in cases:
            for excl in (False, True):
                check_scan(x, op, excl, ops, lvl, g, b)
        # a reversed run whose chunks of four end on 16-byte boundaries (whole 128-bit
        # copies, read last point first), whole and with a ragged end
        x4 = data(op, dtype, 300_004, 54)
        for ops in ([("reverse", 0)], [("split_snd", 777, 0), ("reverse", 0)]):
            for excl in (False, True):
                check_scan(x4, op, excl, ops)


@pytest.mark.parametrize("op", ["argmax", "argmin"])
def test_arg_scan_general_path(op):
    """desc_force_generic: contiguous arg scans through the map form of the
    arg look-back scan (a one-dim map of stride 1, 128-bit copies), plain and
    one segment per block, against the oracle."""
    n = 5 * 8192 + 12
    D.desc_force_generic(True)
    try:
        for dtype in ("i32", "f32"):
            x = data(op, dtype, n, 61)
            for excl in (False, True):
                check_scan(x, op, excl)
                check_scan(x, op, excl, [("group", 4, 0), ("select", V.BLOCK, V.X)], V.BLOCK, (n // 4, 1, 1),
                           (1, 1, 1), seg_len=4)
    finally:
        D.desc_force_generic(False)


@pytest.mark.parametrize("op", ["argmax", "argmin", "sum", "max", "xor"])
def test_scan_reversed_runs_per_block(op):
    """A reversed array grouped per block lowers to one dim of stride -1 with
    a period: per-level segments through the descending 128-bit copies, the
    segment length a multiple of 4 and not, against the oracle."""
    n = 12 * 4100                                        # six 8192-point tiles and a ragged seventh
    for m in (8, 1025, 4100, 4920):
        ops = [("reverse", 0), ("group", m, 0), ("select", V.BLOCK, V.X)]
        for dtype in (("i32", "f32") if op in ("argmax", "argmin", "sum", "max") else ("i32",)):
            x = data(op, dtype, n, 71) if op in INT_OPS else (
                synth.ints_pm1000(n, seed=71) if dtype == "i32" else synth.uniform_grid(n, seed=71))
            for excl in (False, True):
                if op == "sum" and dtype == "f32":
                    got = D.desc_scan(x.cuda(), [n], ops, V.BLOCK, (n // m, 1, 1), (1, 1, 1),
                                      flags=D.EXCLUSIVE if excl else 0).cpu().numpy()
                    want, pa = O.scan_op(x.numpy(), np.zeros(n, np.float32), [n], ops, V.BLOCK, "sum", excl,
                                         (n // m, 1, 1), (1, 1, 1))
                    assert np.all(np.abs(got - want) <= 1e-5 * pa + 1e-30)
                else:
                    check_scan(x, op, excl, ops, V.BLOCK, (n // m, 1, 1), (1, 1, 1), seg_len=m)
