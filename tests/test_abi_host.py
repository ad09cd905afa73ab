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
