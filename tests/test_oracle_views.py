"""Pins of the oracle's view algebra and access-conflict check (CPU only).

Each pin compares the oracle with something other than itself: the paper's
worked examples and verdicts (tests/golden), NumPy's own reshape / swapaxes /
flip / slicing applied to an index array, and algebraic invariants.
"""
import json
import math
import os
import random

import numpy as np
import pytest

from oracle import views as V

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def numpy_eval(base, ops):
    """Independent evaluation: apply each view as a NumPy array operation to
    arange(n).reshape(base); selects keep their axis in front (row-major
    order of the domain puts selected dims first, in select order)."""
    a = np.arange(math.prod(base)).reshape(base)
    nsel = 0
    for op in ops:
        if op[0] == "select":
            nsel += 1
            continue
        ax = nsel + op[-1]
        sl = (slice(None),) * ax
        if op[0] == "group":
            k = op[1]
            a = a.reshape(a.shape[:ax] + (a.shape[ax] // k, k) + a.shape[ax + 1:])
        elif op[0] == "split_fst":
            a = a[sl + (slice(0, op[1]),)]
        elif op[0] == "split_snd":
            a = a[sl + (slice(op[1], None),)]
        elif op[0] == "transpose":
            a = np.swapaxes(a, ax, ax + 1)
        elif op[0] == "reverse":
            a = np.flip(a, axis=ax)
    return a


def random_chain(rng, base, nops, allow_select=True, allow_split=True):
    ops, shape = [], list(base)
    for _ in range(nops):
        choices = []
        for d in range(len(shape)):
            n = shape[d]
            divs = [k for k in range(1, n + 1) if n % k == 0]
            if divs:
                choices.append(("group", rng.choice(divs), d))
            if allow_split:
                choices.append(("split_fst", rng.randint(0, n), d))
                choices.append(("split_snd", rng.randint(0, n), d))
            choices.append(("reverse", d))
            if d + 1 < len(shape):
                choices.append(("transpose", d))
        if allow_select and len(shape) > 1:
            choices.append(("select", V.THREAD, V.X))
        op = rng.choice(choices)
        ops.append(op)
        shape = V.stages(base, ops)[-1]
    return ops


def test_select_view_figure():
    g = json.load(open(os.path.join(GOLD, "select_view_figure.json")))
    ops = [("group", 8, 0), ("transpose", 0), ("select", V.THREAD, V.X)]
    V.check_selects(g["base_shape"], ops, (1, 1, 1), (g["threads"], 1, 1))
    for t, want in enumerate(g["thread_elements"]):
        got = [V.resolve(g["base_shape"], ops, [t], [i]) for i in range(4)]
        assert got == want


@pytest.mark.parametrize("seed", range(200))
def test_resolve_matches_numpy(seed):
    rng = random.Random(seed)
    base = rng.choice([[24], [36], [6, 8], [4, 6, 2], [64], [2, 3, 4, 5]])
    ops = random_chain(rng, base, rng.randint(1, 5))
    want = numpy_eval(base, ops)
    got = V.domain_indices(base, ops)
    assert list(got.shape) == list(want.shape)
    assert np.array_equal(got, want)


def test_types_of_basic_views():
    # listing of basic view types: shapes after each view
    assert V.stages([12], [("group", 4, 0)])[-1] == [3, 4]
    assert V.stages([12], [("split_fst", 5, 0)])[-1] == [5]
    assert V.stages([12], [("split_snd", 5, 0)])[-1] == [7]
    assert V.stages([3, 5], [("transpose", 0)])[-1] == [5, 3]
    assert V.stages([12], [("reverse", 0)])[-1] == [12]
    assert V.stages([4, 6], [("group", 3, 1)])[-1] == [4, 2, 3]        # map(group)
    with pytest.raises(V.ViewError):
        V.stages([12], [("group", 5, 0)])                              # n mod k != 0
    with pytest.raises(V.ViewError):
        V.stages([12], [("split_fst", 13, 0)])                         # n >= k violated
    with pytest.raises(V.ViewError):
        V.stages([12], [("transpose", 0)])                             # needs nesting


def test_involutions_and_identity():
    for base in ([8, 8], [3, 7], [2, 5, 4]):
        n = math.prod(base)
        ident = np.arange(n).reshape(base)
        for d in range(len(base) - 1):
            assert np.array_equal(V.domain_indices(base, [("transpose", d), ("transpose", d)]), ident)
        for d in range(len(base)):
            assert np.array_equal(V.domain_indices(base, [("reverse", d), ("reverse", d)]), ident)
    # group then row-major flatten is the identity
    for n, k in ((12, 3), (64, 8), (30, 1), (30, 30)):
        assert np.array_equal(V.domain_indices([n], [("group", k, 0)]).ravel(), np.arange(n))


@pytest.mark.parametrize("seed", range(50))
def test_chains_without_split_are_permutations(seed):
    rng = random.Random(1000 + seed)
    base = [48]
    ops = random_chain(rng, base, 4, allow_select=False, allow_split=False)
    idx = V.domain_indices(base, ops).ravel()
    assert sorted(idx.tolist()) == list(range(48))


def test_split_halves_partition():
    for n in (1, 7, 64):
        for k in range(n + 1):
            a = V.domain_indices([n], [("split_fst", k, 0)]).ravel().tolist()
            b = V.domain_indices([n], [("split_snd", k, 0)]).ravel().tolist()
            assert not set(a) & set(b)
            assert sorted(a + b) == list(range(n))


def test_select_extent_must_match_resources():
    ops = [("group", 32, 0), ("select", V.BLOCK, V.X), ("select", V.THREAD, V.X)]
    V.check_selects([1024], ops, (32, 1, 1), (32, 1, 1))
    with pytest.raises(V.ViewError):                   # 1024 elements, 64 blocks
        V.check_selects([1024], ops, (64, 1, 1), (32, 1, 1))
    # scale_vec example (Section 2.3): launched with bytes instead of elements
    ops1 = [("select", V.THREAD, V.X)]
    with pytest.raises(V.ViewError):
        V.check_selects([256], ops1, (1, 1, 1), (256 * 8, 1, 1))
    # selection order must narrow: thread before block is rejected
    with pytest.raises(V.ViewError):
        V.check_selects([1024], [("group", 32, 0), ("select", V.THREAD, V.X), ("select", V.BLOCK, V.X)],
                        (32, 1, 1), (32, 1, 1))


def _verdict(name):
    G, Bk = (2, 2, 1), (32, 8, 1)
    if name.startswith("cuda_transpose"):
        # tmp index written by thread (x, y) at iteration j in {0, 8, 16, 24}
        if name.endswith("buggy_tmp_write"):   # y + 32*j + x  with j = 8*i
            ext, st = [32, 8, 4], [1, 1, 256]
        else:                                  # x + 32*(y + j)
            ext, st = [32, 8, 4], [1, 32, 256]
        binds = [("thread", V.X), ("thread", V.Y), ("local",)]
        # shared memory is per block: one buffer per block index
        acc = []
        for b in range(4):
            t, e = V.affine_access(ext, st, 0, binds, (1, 1, 1), Bk)
            acc.append((b, t, e, True))
        return V.first_conflict(acc)
    if name == "rev_per_block":
        n, B = 256, 64
        w = (0, [n], [("group", B, 0), ("select", V.BLOCK, V.X), ("select", V.THREAD, V.X)], True)
        r = (0, [n], [("group", B, 0), ("select", V.BLOCK, V.X), ("reverse", 0), ("select", V.THREAD, V.X)], False)
        return V.views_disjoint([w, r], (4, 1, 1), (B, 1, 1))
    g, b = (32, 1, 1), (32, 1, 1)
    if name == "narrowing_line4_uniq_whole_array_per_block":
        return V.views_disjoint([(0, [1024], [], True)], g, b)
    if name == "narrowing_line6_group_thread_without_block":
        return V.views_disjoint([(0, [1024], [("group", 32, 0), ("select", V.THREAD, V.X)], True)], g, b)
    if name == "narrowing_line8_group_block_thread":
        return V.views_disjoint([(0, [1024], [("group", 32, 0), ("select", V.BLOCK, V.X),
                                              ("select", V.THREAD, V.X)], True)], g, b)
    g, b = (1, 1, 1), (32, 1, 1)
    fst = [("split_fst", 32, 0), ("select", V.THREAD, V.X)]
    snd = [("split_snd", 32, 0), ("select", V.THREAD, V.X)]
    if name == "split_fst_vs_snd":
        return V.views_disjoint([(0, [64], fst, True), (0, [64], snd, True)], g, b)
    if name == "split_fst_vs_whole":
        whole = [("group", 2, 0), ("select", V.THREAD, V.X)]
        return V.views_disjoint([(0, [64], fst, True), (0, [64], whole, False)], g, b)
    raise KeyError(name)


def test_paper_verdicts():
    g = json.load(open(os.path.join(GOLD, "paper_verdicts.json")))
    for case in g["cases"]:
        got = _verdict(case["name"])
        assert (got is None) == (case["verdict"] == "accept"), case["name"]


def test_buggy_transpose_collision_is_the_expected_pair():
    # (x=1, y=0) and (x=0, y=1) both write tmp[1] at j=0 in the buggy index
    t, e = V.affine_access([32, 8, 4], [1, 1, 256], 0, [("thread", V.X), ("thread", V.Y), ("local",)],
                           (1, 1, 1), (32, 8, 1))
    assert V.first_conflict([(0, t, e, True)]) == 1


def test_warp_and_lane_binding():
    # group(32)[[warp]][[thread]] inside one block of 128 threads: lane l of warp w gets 32 w + l
    ops = [("group", 32, 0), ("select", V.WARP, V.X), ("select", V.THREAD, V.X)]
    t, e = V.view_access([128], ops, (1, 1, 1), (128, 1, 1))
    assert np.array_equal(np.sort(e), np.arange(128))
    assert np.array_equal(e[np.argsort(t)], np.arange(128))
    assert V.views_disjoint([(0, [128], ops, True)], (1, 1, 1), (128, 1, 1)) is None
