"""desc_check_program (C ABI, host only) against the oracle: the pinned
programs of test_oracle_program and random programs of accesses, barriers
and splits (status, statement index and first conflicting element)."""
import random

import pytest

import paper_2305_03448_gb300 as D
import test_oracle_program as T
from oracle import program as P
from oracle.views import BLOCK, GRID, THREAD, WARP, X

PINNED = [
    ([("split", THREAD, X, 32, [("sync", BLOCK)], [])], (1, 1, 1), (64, 1, 1)),
    ([("access", 0, [64], [("reverse", 0), ("select", THREAD, X)], False),
      ("access", 0, [64], [("select", THREAD, X)], True)], (1, 1, 1), (64, 1, 1)),
    ([("access", 0, [1024], [("group", 32, 0), ("select", THREAD, X)], True)], (32, 1, 1), (32, 1, 1)),
    ([("access", 0, [64], [("group", 32, 0), ("select", BLOCK, X), ("select", THREAD, X)], True), ("sync", BLOCK),
      ("access", 0, [64], [("group", 32, 0), ("reverse", 0), ("select", BLOCK, X), ("select", THREAD, X)], False)],
     (2, 1, 1), (32, 1, 1)),
    ([("split", WARP, X, 1, [("sync", BLOCK)], [])], (1, 1, 1), (128, 1, 1)),
    ([("split", THREAD, 1, 2, [("access", 0, [2, 16], [("select", THREAD, 1), ("select", THREAD, X)], True)],
       [("access", 0, [2, 16], [("select", THREAD, 1), ("select", THREAD, X)], True)])], (1, 1, 1), (16, 4, 1)),
]


@pytest.mark.parametrize("case", range(len(PINNED)))
def test_pinned_programs_match_oracle(desc_lib, case):
    prog, g, b = PINNED[case]
    assert D.desc_check_program(prog, g, b) == P.check_program(prog, g, b)


def test_oracle_pins_module_is_present():
    assert hasattr(T, "test_section_2_2_barrier_inside_split_block")


def _views(rng, sub, L):
    """A random view of an L-element buffer whose selects fit the 1-D sub-resource."""
    nbx, ntx, warps = sub["nb"], sub["nt"], sub["nw"]
    modes = ["thread", "block_thread", "whole", "thread_local"] if ntx else ["whole"]
    if warps:
        modes.append("lanes")
    mode = rng.choice(modes)
    if mode == "thread":
        n = ntx
        sel = [("select", THREAD, X)]
    elif mode == "block_thread":
        n = nbx * ntx
        sel = [("group", ntx, 0), ("select", BLOCK, X), ("select", THREAD, X)]
    elif mode == "thread_local":
        n = 2 * ntx
        sel = [("group", 2, 0), ("select", THREAD, X)]
    elif mode == "lanes":
        n = warps * 32
        sel = [("group", 32, 0), ("select", WARP, X), ("select", THREAD, X)]
    else:
        n = rng.choice([1, 7, 32])
        sel = []
    if n > L:
        return None
    off = rng.randrange(0, L - n + 1)
    ops = []
    if off:
        ops.append(("split_snd", off, 0))
    if off + n < L:
        ops.append(("split_fst", n, 0))
    if rng.random() < 0.4:
        ops.append(("reverse", 0))
    return ops + sel


def _program(rng, sub, L, depth, budget):
    out = []
    for _ in range(rng.randint(1, 4)):
        if budget[0] <= 0:
            break
        budget[0] -= 1
        r = rng.random()
        if r < 0.55:
            ops = _views(rng, sub, L)
            if ops is None:
                continue
            out.append(("access", rng.randrange(2), [L], ops, rng.random() < 0.5))
        elif r < 0.75:
            out.append(("sync", rng.choice([BLOCK, BLOCK, WARP, GRID])))
        elif depth < 2:
            level = rng.choice([BLOCK, THREAD, WARP])
            if level == BLOCK and sub["nb"] > 1:
                at = rng.randrange(1, sub["nb"])
                a = dict(sub, nb=at)
                b = dict(sub, nb=sub["nb"] - at)
            elif level == THREAD and sub["nt"] > 1 and not sub["warp_split"]:
                at = rng.randrange(1, sub["nt"])
                a = dict(sub, nt=at, nw=0)
                b = dict(sub, nt=sub["nt"] - at, nw=0)
            elif level == WARP and sub["nw"] > 1:
                at = rng.randrange(1, sub["nw"])
                a = dict(sub, nw=at, nt=0, warp_split=True)
                b = dict(sub, nw=sub["nw"] - at, nt=0, warp_split=True)
            else:
                continue
            out.append(("split", level, X, at, _program(rng, a, L, depth + 1, budget),
                        _program(rng, b, L, depth + 1, budget)))
    return out


def test_random_programs_match_oracle(desc_lib):
    rng = random.Random(2305)
    seen = set()
    for _ in range(250):
        nb = rng.choice([1, 2, 3])
        nt = rng.choice([32, 64, 96])
        g, b = (nb, 1, 1), (nt, 1, 1)
        L = rng.choice([64, 200, 400])
        sub = {"nb": nb, "nt": nt, "nw": nt // 32, "warp_split": False}
        prog = _program(rng, sub, L, 0, [8])
        want = P.check_program(prog, g, b)
        got = D.desc_check_program(prog, g, b)
        assert got == want, (prog, g, b)
        seen.add(want[0])
    assert {0, 3, 11} <= seen
