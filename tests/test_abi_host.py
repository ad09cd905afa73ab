"""The C ABI on the host (no GPU): every declared symbol is exported, view
lowering matches the oracle's view interpreter point by point, and the
access-conflict check matches the oracle's enumeration."""
import glob
import math
import os
import random
import re

import numpy as np
import pytest

import paper_2305_03448_gb300 as D
from oracle import views as V

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(desc_\w+)\s*\([^;{]*\)\s*;", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(desc_lib):
    names = declared_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(desc_lib, n)]
    assert not missing, missing


def test_status_strings_and_version(desc_lib):
    for code, name in D.STATUS.items():
        assert desc_lib.desc_status_string(code).decode() == name
    assert desc_lib.desc_version() >> 16 == 1


def c_map_elements(m):
    """Evaluate the lowered affine map over its domain (row-major)."""
    ext = m["extent"]
    if not ext:
        return np.array(m["offset"])
    idx = np.indices(ext, dtype=np.int64) if all(ext) else np.zeros([len(ext)] + ext, np.int64)
    return m["offset"] + sum(idx[i] * m["stride"][i] for i in range(len(ext)))


def random_view(rng):
    base = rng.choice([[24], [36], [6, 8], [4, 6, 2], [64], [2, 3, 4, 5], [48]])
    ops, shape, nsel = [], list(base), 0
    for _ in range(rng.randint(0, 6)):
        choices = []
        for d in range(len(shape)):
            n = shape[d]
            divs = [k for k in range(1, n + 1) if n % k == 0]
            if divs:
                choices.append(("group", rng.choice(divs), d))
            choices += [("split_fst", rng.randint(0, n), d), ("split_snd", rng.randint(0, n), d), ("reverse", d)]
            if d + 1 < len(shape):
                choices.append(("transpose", d))
        if len(shape) > 1 and nsel < 3:
            choices.append(("select", V.THREAD, nsel))      # each (level, dim) once
        op = rng.choice(choices)
        nsel += op[0] == "select"
        ops.append(op)
        shape = V.stages(base, ops)[-1]
    return base, ops


@pytest.mark.parametrize("seed", range(300))
def test_lowering_matches_oracle_interpreter(desc_lib, seed):
    base, ops = random_view(random.Random(seed))
    m = D.desc_lower_view(base, ops)
    assert m["base_elems"] == math.prod(base)
    want = V.domain_indices(base, ops)
    got = c_map_elements(m)
    assert list(np.shape(got)) == list(want.shape)
    assert np.array_equal(got, want)


def test_lowering_of_the_transpose_listing_views(desc_lib):
    # input.group_by_tile-like view: 2-D tiles selected by blocks (Y, X),
    # each tile's rows grouped 8 at a time and transposed (thread (x, y),
    # item i -> tile element (y + 8 i, x)), for a 64 x 64 matrix
    base = [64, 64]
    ops = [("group", 32, 0), ("group", 32, 2), ("transpose", 1),          # [2][2][32][32] tiles
           ("select", V.BLOCK, V.Y), ("select", V.BLOCK, V.X),
           ("group", 8, 0), ("transpose", 0), ("transpose", 1),            # [8][32][4]
           ("select", V.THREAD, V.Y), ("select", V.THREAD, V.X)]
    grid, block = (2, 2, 1), (32, 8, 1)
    m = D.desc_lower_view(base, ops, grid, block)
    assert np.array_equal(c_map_elements(m), V.domain_indices(base, ops))
    # thread (x=3, y=2) of block (x=1, y=0), item 1: row 2 + 8, col 32 + 3
    e = m["offset"] + sum(c * s for c, s in zip([0, 1, 2, 3, 1], m["stride"]))
    assert e == (2 + 8) * 64 + 32 + 3
    assert V.views_disjoint([(0, base, ops, True)], grid, block) is None


@pytest.mark.parametrize("bad", [
    ([12], [("group", 5, 0)]),                       # n mod k != 0
    ([12], [("split_fst", 13, 0)]),                  # split beyond the extent
    ([12], [("transpose", 0)]),                      # not nested
    ([12], [("reverse", 1)]),                        # depth out of range
    ([4, 8], [("select", V.THREAD, V.X), ("select", V.BLOCK, V.X)]),   # does not narrow
])
def test_lowering_rejects_ill_typed_views(desc_lib, bad):
    with pytest.raises(D.DescError) as e:
        D.desc_lower_view(*bad)
    assert e.value.status == 2


def test_select_extent_checked_against_exec(desc_lib):
    ops = [("group", 32, 0), ("select", V.BLOCK, V.X), ("select", V.THREAD, V.X)]
    D.desc_lower_view([1024], ops, (32, 1, 1), (32, 1, 1))
    with pytest.raises(D.DescError) as e:
        D.desc_lower_view([1024], ops, (64, 1, 1), (32, 1, 1))
    assert e.value.status == 2
    # launched with bytes instead of elements (Section 2.3)
    with pytest.raises(D.DescError):
        D.desc_lower_view([256], [("select", V.THREAD, V.X)], (1, 1, 1), (256 * 4, 1, 1))


# ------------------------------------------------------------- disjointness
def _c_verdict_views(accesses, grid, block):
    acc = [(D.desc_lower_view(shape, ops, grid, block), buf, w) for buf, shape, ops, w in accesses]
    return D.desc_check_disjoint(acc, grid, block)


def test_paper_verdicts_through_the_abi(desc_lib):
    g, b = (32, 1, 1), (32, 1, 1)
    full = [("group", 32, 0), ("select", V.BLOCK, V.X), ("select", V.THREAD, V.X)]
    assert _c_verdict_views([(0, [1024], full, True)], g, b) is None   # narrowed to one element per thread: accept
    assert _c_verdict_views([(0, [1024], [], True)], g, b) == 0        # the whole array written by every thread
    assert _c_verdict_views([(0, [1024], [("group", 32, 0), ("select", V.THREAD, V.X)], True)], g, b) == 0
    n, B = 256, 64
    w = (0, [n], [("group", B, 0), ("select", V.BLOCK, V.X), ("select", V.THREAD, V.X)], True)
    r = (0, [n], [("group", B, 0), ("select", V.BLOCK, V.X), ("reverse", 0), ("select", V.THREAD, V.X)], False)
    assert _c_verdict_views([w, r], (4, 1, 1), (B, 1, 1)) == V.views_disjoint(
        [(0, [n], w[2], True), (0, [n], r[2], False)], (4, 1, 1), (B, 1, 1))
    fst = [("split_fst", 32, 0), ("select", V.THREAD, V.X)]
    snd = [("split_snd", 32, 0), ("select", V.THREAD, V.X)]
    assert _c_verdict_views([(0, [64], fst, True), (0, [64], snd, True)], (1, 1, 1), (32, 1, 1)) is None


def test_cuda_transpose_listing_indices(desc_lib):
    """The shared-memory write index of the Section 1 listing as a raw map."""
    def raw(strides):
        return {"ndims": 3, "nsel": 2, "extent": [8, 32, 4], "stride": strides,
                "level": [V.THREAD, V.THREAD, -1], "dim": [V.Y, V.X, -1], "offset": 0}
    bk = (32, 8, 1)
    assert D.desc_check_disjoint([(raw([1, 1, 256]), 0, True)], (1, 1, 1), bk) == 1      # buggy
    assert D.desc_check_disjoint([(raw([32, 1, 256]), 0, True)], (1, 1, 1), bk) is None  # fixed


def _random_ops(rng, n, grid, block):
    """A random chain that selects blocks (Y, X) and threads (Y, X) over an
    array of n = grid * block * r elements, with optional reverses, or
    selects nothing at all."""
    ops, m = [], n
    if rng.random() < 0.8:
        ops += [("group", m // grid[1], 0), ("select", V.BLOCK, V.Y)]
        m //= grid[1]
        if rng.random() < 0.3:
            ops.append(("reverse", 0))
        ops += [("group", m // grid[0], 0), ("select", V.BLOCK, V.X)]
        m //= grid[0]
    if rng.random() < 0.8:
        ops += [("group", m // block[1], 0), ("select", V.THREAD, V.Y)]
        m //= block[1]
        if rng.random() < 0.3:
            ops.append(("reverse", 0))
        ops += [("group", m // block[0], 0), ("select", V.THREAD, V.X)]
    return ops


@pytest.mark.parametrize("seed", range(150))
def test_disjointness_matches_oracle(desc_lib, seed):
    rng = random.Random(7000 + seed)
    grid = (rng.choice([1, 2, 3]), rng.choice([1, 2]), 1)
    block = (rng.choice([1, 2, 4, 32]), rng.choice([1, 2]), 1)
    gb = grid[0] * grid[1] * block[0] * block[1]
    sizes = {0: gb * rng.choice([1, 2, 3]), 1: gb * rng.choice([1, 2])}
    accesses = []
    for _ in range(rng.randint(1, 3)):
        buf = rng.choice([0, 0, 1])
        accesses.append((buf, [sizes[buf]], _random_ops(rng, sizes[buf], grid, block), rng.random() < 0.6))
    want = V.views_disjoint(accesses, grid, block)
    got = _c_verdict_views(accesses, grid, block)
    assert got == want


# ------------------------------------------------ disjointness: the wider sweep
# Views over 1-, 2- and 3-D base arrays with group, split (fst / snd),
# transpose and reverse at any nesting depth, selected by blocks (X, Y),
# warps and lanes or threads (X, Y), with unselected execution dims that
# replicate the access; several accesses per buffer, some built to overlap
# (a split half written beside the whole, a read through a reversed view);
# and raw affine maps whose strides may repeat, vanish or change sign.
_BASES = [[64], [96], [8, 16], [4, 6, 8], [2, 64], [32, 32], [3, 4, 32], [128, 4], [6, 10], [64, 3], [2, 2, 64],
          [5, 7], [36]]


def _rand_view_op(rng, shape):
    """One random non-select view op valid for `shape` (or None)."""
    choices = []
    for d in range(len(shape)):
        n = shape[d]
        divs = [k for k in range(1, n + 1) if n % k == 0]
        if divs:
            choices.append(("group", rng.choice(divs), d))
        choices += [("split_fst", rng.randint(0, n), d), ("split_snd", rng.randint(0, n), d), ("reverse", d)]
        if d + 1 < len(shape):
            choices.append(("transpose", d))
    return rng.choice(choices) if choices else None


def _selected_view(rng, base):
    """A random chain over `base` whose selects narrow block -> warp / lane or
    thread, with view ops before, between and after them."""
    ops, shape = [], list(base)

    def some_ops(k):
        nonlocal shape
        for _ in range(rng.randint(0, k)):
            op = _rand_view_op(rng, shape)
            if op is None or len(shape) > 5:
                return
            ops.append(op)
            shape = V.stages(base, ops)[-1]

    some_ops(3)
    levels = []
    if rng.random() < 0.7:
        levels += rng.sample([(V.BLOCK, V.Y), (V.BLOCK, V.X)], rng.randint(1, 2))
    r = rng.random()
    if r < 0.3:
        levels += [(V.WARP, V.X)] + ([(V.THREAD, V.X)] if rng.random() < 0.7 else [])
    elif r < 0.8:
        levels += rng.sample([(V.THREAD, V.Y), (V.THREAD, V.X)], rng.randint(1, 2))
    warp = False
    for lvl, dim in levels:
        some_ops(1)
        if not shape:
            break
        lane = lvl == V.THREAD and warp
        if lane and shape[0] != 32:
            if shape[0] > 0 and shape[0] % 32 == 0:     # bring 32 lanes outermost
                ops.append(("group", shape[0] // 32, 0))
                ops.append(("transpose", 0))
                shape = V.stages(base, ops)[-1]
            else:
                break
        if shape[0] > 64 and not lane:
            continue                                    # keep the resource counts small
        ops.append(("select", lvl, dim))
        warp = warp or lvl == V.WARP
        shape = V.stages(base, ops)[-1]
    some_ops(2)
    return ops


def _exec_for(rng, base, ops):
    """The execution resource whose counts match the view's selects; the
    dims it does not select get small random extents (replication)."""
    grid, block = [1, 1, 1], [1, 1, 1]
    sels = V.selects(base, ops)
    warp_e, lane = None, False
    for lvl, dim, e in sels:
        if lvl == V.BLOCK:
            grid[dim] = e
        elif lvl == V.WARP:
            warp_e = e
        elif warp_e is not None:
            lane = True
        else:
            block[dim] = e
    bsel = {d for lvl, d, _ in sels if lvl == V.BLOCK}
    tsel = {d for lvl, d, _ in sels if lvl == V.THREAD}
    for d in range(2):
        if d not in bsel and rng.random() < 0.3:
            grid[d] = rng.choice([2, 3])
    if warp_e is not None or (lane and warp_e is None):
        block = [32 * (warp_e if warp_e is not None else rng.choice([1, 2])), 1, 1]
    else:
        for d in range(2):
            if d not in tsel and rng.random() < 0.3:
                block[d] = rng.choice([2, 4])
    return tuple(grid), tuple(block)


def _wide_case(seed):
    """(accesses, grid, block) or None when the draw is not a valid program."""
    rng = random.Random(91000 + seed)
    base = rng.choice(_BASES)
    try:
        ops = _selected_view(rng, base)
        grid, block = _exec_for(rng, base, ops)
    except V.ViewError:
        return None
    acc = [(0, base, ops, True)]
    r = rng.random()
    if r < 0.2:                                         # a split half written beside the whole
        k = rng.randint(1, base[0])
        acc.append((0, base, [("split_fst", k, 0)], True))
    elif r < 0.45:                                      # a read of the same buffer through other views
        acc.append((0, base, ops[:-1] + [("reverse", 0)] if ops and ops[-1][0] != "select" and
                    V.stages(base, ops)[-1] else [("reverse", 0)], False))
    elif r < 0.6:                                       # a second buffer, written through its own view
        b2 = rng.choice(_BASES)
        acc.append((1, b2, _selected_view(rng, b2), True))
    try:
        for _, b, o, _ in acc:
            V.check_selects(b, o, grid, block)
    except V.ViewError:
        return None
    if math.prod(grid) * math.prod(block) > 1024 or 0 in grid or 0 in block:
        return None                                     # an empty resource is not a launch
    return acc, grid, block


def test_disjointness_wide_sweep_matches_oracle(desc_lib):
    stats = {"accept": 0, "reject": 0, "structural_accept": 0, "structural_reject": 0, "enumerated": 0,
             "warp": 0, "transpose": 0, "split": 0, "multi_reverse": 0, "replicated": 0, "2d3d": 0}
    cases, seed = 0, 0
    while cases < 600:
        c = _wide_case(seed)
        seed += 1
        if c is None:
            continue
        acc, grid, block = c
        want = V.views_disjoint(acc, grid, block)
        got, how = _c_verdict_views_method(acc, grid, block)
        assert got == want, (seed - 1, acc, grid, block)
        cases += 1
        ops = acc[0][2]
        stats["accept" if want is None else "reject"] += 1
        if how == D.DECIDED_STRUCTURAL:
            stats["structural_accept" if want is None else "structural_reject"] += 1
        if how & D.DECIDED_ENUMERATION:
            stats["enumerated"] += 1
        stats["warp"] += any(o[0] == "select" and o[1] == V.WARP for o in ops)
        stats["transpose"] += any(o[0] == "transpose" for o in ops)
        stats["split"] += any(o[0].startswith("split") for o in ops)
        stats["multi_reverse"] += len({o[1] for o in ops if o[0] == "reverse"}) > 1
        stats["replicated"] += any(g > 1 for g in grid[:2]) and len(
            [o for o in ops if o[0] == "select" and o[1] == V.BLOCK]) < sum(g > 1 for g in grid[:2])
        stats["2d3d"] += len(acc[0][1]) > 1
    print(stats)
    assert stats["accept"] >= 100 and stats["reject"] >= 100
    assert stats["structural_accept"] >= 100 and stats["structural_reject"] >= 20
    assert stats["enumerated"] >= 50
    for k in ("warp", "transpose", "split", "multi_reverse", "replicated", "2d3d"):
        assert stats[k] >= 20, (k, stats)


def _c_verdict_views_method(accesses, grid, block):
    acc = [(D.desc_lower_view(shape, ops, grid, block), buf, w) for buf, shape, ops, w in accesses]
    return D.desc_check_disjoint(acc, grid, block, with_method=True)


_BINDS = [("block", V.X), ("block", V.Y), ("thread", V.X), ("thread", V.Y), ("local",), ("local",)]


def _raw_case(rng):
    """A raw affine write map (and sometimes a read map) with random strides."""
    grid = (rng.choice([1, 2, 3]), rng.choice([1, 2]), 1)
    block = (rng.choice([1, 2, 4, 8]), rng.choice([1, 2]), 1)
    nd = rng.randint(1, 4)
    binds = rng.sample(_BINDS, nd)
    ext, stride = [], []
    for b in binds:
        if b[0] == "block":
            ext.append(grid[b[1]] if rng.random() < 0.85 else grid[b[1]] + 1)
        elif b[0] == "thread":
            ext.append(block[b[1]] if rng.random() < 0.85 else max(1, block[b[1]] - 1))
        else:
            ext.append(rng.randint(1, 5))
    if rng.random() < 0.5:                              # row-major strides of a permutation: injective
        order = list(range(nd))
        rng.shuffle(order)
        c = 1
        stride = [0] * nd
        for i in reversed(order):
            stride[i] = c * rng.choice([1, -1])
            c *= ext[i]
    else:                                               # small strides: repeats, zeros, sign changes
        stride = [rng.randint(-6, 6) for _ in range(nd)]
    off = sum(max(0, -s) * (e - 1) for s, e in zip(stride, ext)) + rng.randint(0, 3)
    return grid, block, binds, ext, stride, off


def _lowered_of_raw(binds, ext, stride, off):
    sel = [i for i, b in enumerate(binds) if b[0] != "local"]
    loc = [i for i, b in enumerate(binds) if b[0] == "local"]
    order = sel + loc
    lvl = {"block": V.BLOCK, "thread": V.THREAD}
    return {"ndims": len(order), "nsel": len(sel), "extent": [ext[i] for i in order],
            "stride": [stride[i] for i in order],
            "level": [lvl[binds[i][0]] if binds[i][0] != "local" else -1 for i in order],
            "dim": [binds[i][1] if binds[i][0] != "local" else -1 for i in order], "offset": off}


@pytest.mark.parametrize("seed", range(400))
def test_disjointness_raw_maps_match_oracle(desc_lib, seed):
    rng = random.Random(123000 + seed)
    grid, block, binds, ext, stride, off = _raw_case(rng)
    # the oracle's binds: ("block", dim), ("thread", dim), ("local",)
    t, e = V.affine_access(ext, stride, off, binds, grid, block)
    acc_o = [(0, t, e, True)]
    acc_c = [(_lowered_of_raw(binds, ext, stride, off), 0, True)]
    if rng.random() < 0.4:                              # a read map beside it
        g2, b2, bi2, ex2, st2, of2 = _raw_case(rng)
        bi2 = [b if b[0] == "local" or (b[0] == "block" and ex2[i] <= grid[b[1]]) or
               (b[0] == "thread" and ex2[i] <= block[b[1]]) else ("local",) for i, b in enumerate(bi2)]
        t2, e2 = V.affine_access(ex2, st2, of2, bi2, grid, block)
        acc_o.append((0, t2, e2, False))
        acc_c.append((_lowered_of_raw(bi2, ex2, st2, of2), 0, False))
    want = V.first_conflict(acc_o)
    got = D.desc_check_disjoint(acc_c, grid, block)
    assert got == want, (grid, block, binds, ext, stride, off)
