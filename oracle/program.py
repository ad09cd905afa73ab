"""Oracle: access safety across a kernel body (test infrastructure only).

Section 3.3 ("Narrowing", "Synchronization") and Section 4
(access_safety_check): the type checker keeps an environment of which
execution resource accessed which place; a barrier removes the entries of the
threads it synchronises.  Section 2.2 ("Synchronization") rejects a barrier
that some thread of its block does not reach: a sync inside a split of the
block's threads.

A program is a list of statements run by the current (sub-)resource:
  ("access", buffer, base_shape, ops, is_write)
  ("sync", level)          BLOCK: all threads of each block of the resource;
                           WARP: each warp; GRID: a kernel boundary
  ("split", level, dim, at, first, second)
                           BLOCK: the blocks along dim; THREAD: each block's
                           threads along dim; WARP: each block's warps (dim X).
                           `first` runs on coordinates < at, `second` on the
                           rest, with coordinates counted from `at`; both run
                           concurrently.
A view's selects bind coordinates relative to the sub-resource, and each
select's extent must equal the sub-resource's count along it.

Readings (the paper gives the rules, not a sub-resource model for warps):
  - the warp of a thread is lin // 32, lin = x + X (y + Y z); warp and lane
    coordinates are undefined where a block's threads are split (THREAD), and
    thread coordinates are undefined where its warps are split (WARP);
  - a BLOCK sync inside a THREAD or WARP split, a WARP sync inside a THREAD
    split or with a thread count that is not a multiple of 32, and a GRID sync
    inside any split are rejected (status 11, the sync's index);
  - conflict (status 3): the same element of the same buffer reached by two
    threads, at least one writing, with no barrier since the earlier access
    that synchronises both (a BLOCK sync of their common block, or a WARP sync
    of their common warp); the reported element is the smallest conflicting
    one of the first access statement (preorder index) that has a conflict;
  - split positions outside (0, extent) and select extents that do not match
    the sub-resource give status 2.
Returns (status, statement index or -1, element or None).
"""
from __future__ import annotations

import itertools

import numpy as np

from .views import BLOCK, GRID, THREAD, WARP, resolve, selects, stages

LANE = 3


class _Stop(Exception):
    def __init__(self, status, index, elem=None):
        super().__init__(status)
        self.status, self.index, self.elem = status, index, elem


def _count(sub, block, level, dim):
    nt = block[0] * block[1] * block[2]
    if level == BLOCK:
        return sub["bh"][dim] - sub["bl"][dim]
    if level == WARP:
        if sub["tsplit"]:
            return None
        return sub["wh"] - sub["wl"] if sub["wsplit"] else nt // 32
    if dim == LANE:
        return None if sub["tsplit"] else 32
    if sub["wsplit"]:
        return None
    return sub["th"][dim] - sub["tl"][dim]


def check_program(prog, grid, block):
    nt = block[0] * block[1] * block[2]
    nw = (nt + 31) // 32
    env = {}                       # (buffer, element) -> [(tid, write, block count, warp count)]
    bsync = {}                     # block -> barriers passed
    wsync = {}                     # (block, warp) -> barriers passed
    counter = [0]

    def block_lin(c):
        return c[0] + grid[0] * (c[1] + grid[1] * c[2])

    def threads(sub):
        """(block id, linear thread id, block coords rel., thread coords rel.)"""
        for bc in itertools.product(*[range(sub["bl"][d], sub["bh"][d]) for d in (2, 1, 0)]):
            bz, by, bx = bc
            b = block_lin((bx, by, bz))
            brel = (bx - sub["bl"][0], by - sub["bl"][1], bz - sub["bl"][2])
            for t in range(nt):
                tc = (t % block[0], (t // block[0]) % block[1], t // (block[0] * block[1]))
                if sub["wsplit"]:
                    if not (sub["wl"] <= t // 32 < sub["wh"]):
                        continue
                elif not all(sub["tl"][d] <= tc[d] < sub["th"][d] for d in range(3)):
                    continue
                trel = tuple(tc[d] - sub["tl"][d] for d in range(3))
                yield b, t, brel, trel

    def access(st, sub, index):
        _, buf, shape, ops, w = st
        sel, after_warp = [], False
        for level, dim, ext in selects(shape, ops):   # a THREAD select after a WARP one binds the lane
            sel.append((level, LANE if (level == THREAD and after_warp) else dim, ext))
            after_warp = after_warp or level == WARP
        for level, dim, ext in sel:
            if ext != _count(sub, block, level, dim):
                raise _Stop(2, index)
        local = stages(shape, ops)[-1]
        if any(e == 0 for e in local) or any(e == 0 for _, _, e in sel):
            return
        lgrid = [g.ravel() for g in np.indices(local, dtype=np.int64)] if local else []
        bad = []
        for b, t, brel, trel in threads(sub):
            coords = []
            reach = True
            for level, dim, ext in sel:
                if level == BLOCK:
                    c = brel[dim]
                elif level == WARP:
                    c = t // 32 - (sub["wl"] if sub["wsplit"] else 0)
                elif dim == LANE:
                    c = t % 32
                else:
                    c = trel[dim]
                if c >= ext:
                    reach = False
                coords.append(c)
            if not reach:
                continue
            elems = np.atleast_1d(np.asarray(resolve(shape, ops, coords, lgrid), dtype=np.int64))
            tid = b * nt + t
            for e in elems.tolist():
                lst = env.setdefault((buf, e), [])
                for (t1, w1, bs1, ws1) in lst:
                    if t1 == tid or not (w1 or w):
                        continue
                    same_block = t1 // nt == b
                    if same_block and bsync.get(b, 0) > bs1:
                        continue
                    if same_block and (t1 % nt) // 32 == t // 32 and wsync.get((b, t // 32), 0) > ws1:
                        continue
                    bad.append(e)
                    break
                lst.append((tid, bool(w), bsync.get(b, 0), wsync.get((b, t // 32), 0)))
        if bad:
            raise _Stop(3, index, min(bad))

    def sync(st, sub, index):
        level = st[1]
        if level == GRID:
            if sub["insplit"]:
                raise _Stop(11, index)
            env.clear()
            return
        blocks = [block_lin((bx, by, bz)) for bz in range(sub["bl"][2], sub["bh"][2])
                  for by in range(sub["bl"][1], sub["bh"][1]) for bx in range(sub["bl"][0], sub["bh"][0])]
        if level == BLOCK:
            if sub["tsplit"] or sub["wsplit"]:
                raise _Stop(11, index)
            for b in blocks:
                bsync[b] = bsync.get(b, 0) + 1
            return
        if level == WARP:
            if sub["tsplit"] or nt % 32:
                raise _Stop(11, index)
            ws = range(sub["wl"], sub["wh"]) if sub["wsplit"] else range(nw)
            for b in blocks:
                for wi in ws:
                    wsync[(b, wi)] = wsync.get((b, wi), 0) + 1
            return
        raise ValueError("sync level")

    def run(stmts, sub):
        for st in stmts:
            index = counter[0]
            counter[0] += 1
            if st[0] == "access":
                access(st, sub, index)
            elif st[0] == "sync":
                sync(st, sub, index)
            elif st[0] == "split":
                _, level, dim, at, first, second = st
                a = {k: (list(v) if isinstance(v, (list, tuple)) else v) for k, v in sub.items()}
                b = {k: (list(v) if isinstance(v, (list, tuple)) else v) for k, v in sub.items()}
                a["insplit"] = b["insplit"] = True
                if level in (BLOCK, THREAD):
                    lo_k, hi_k = ("bl", "bh") if level == BLOCK else ("tl", "th")
                    if level == THREAD and sub["wsplit"]:
                        raise _Stop(2, index)
                    lo, hi = sub[lo_k][dim], sub[hi_k][dim]
                    if not 0 < at < hi - lo:
                        raise _Stop(2, index)
                    a[hi_k][dim] = lo + at
                    b[lo_k][dim] = lo + at
                    if level == THREAD:
                        a["tsplit"] = b["tsplit"] = True
                elif level == WARP:
                    if sub["tsplit"] or nt % 32:
                        raise _Stop(2, index)
                    lo, hi = (sub["wl"], sub["wh"]) if sub["wsplit"] else (0, nw)
                    if not 0 < at < hi - lo:
                        raise _Stop(2, index)
                    a["wsplit"] = b["wsplit"] = True
                    a["wl"], a["wh"], b["wl"], b["wh"] = lo, lo + at, lo + at, hi
                else:
                    raise ValueError("split level")
                run(first, a)
                run(second, b)
            else:
                raise ValueError(st[0])

    top = {"bl": [0, 0, 0], "bh": list(grid), "tl": [0, 0, 0], "th": list(block), "wl": 0, "wh": nw,
           "tsplit": False, "wsplit": False, "insplit": False}
    try:
        run(prog, top)
    except _Stop as s:
        return s.status, s.index, s.elem
    return 0, -1, None
