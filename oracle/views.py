"""Oracle: the view algebra and the access-conflict check (test infrastructure).

Views (Section 3.2, "Views", and the listing of basic view types):
  split<k>   [[d; n]] -> ([[d; k]], [[d; n-k]]), requires n >= k; .fst keeps
             coordinates below k, .snd the coordinates from k on
  group<k>   [[d; n]] -> [[ [[d; k]]; n/k ]]: consecutive runs of k elements
             become the inner arrays (the divisibility clause is cut off in
             the source; it is read as n mod k == 0)
  transpose  [[ [[d; n]]; m ]] -> [[ [[d; m]]; n ]]
  reverse    [[d; n]] -> [[d; n]], element i is input element n-1-i
  map(v)     v applied to every element; here an op carries a depth, and an op
             at depth d acts on the arrays nested d levels deep
Select p[[e]] (Section 3.2, "Place Expressions"): the outermost dimension is
distributed over the sub-resources of e, one element each, so its extent must
equal their number.

Index generation (Section 5, "Code Generation"): a selection through a chain of
views is turned into one raw index by transforming the index view by view,
starting with the view applied last.  ``resolve`` does exactly that, on Python
ints or on NumPy index arrays alike.

Execution resources (Section 3.1; Figure "Execution Resources and Dimensions"):
a grid of blocks (X, Y, Z) of threads (X, Y, Z).  The warp level is not in the
paper; it is read as 32 consecutive linear thread ids, lin = x + X*(y + Y*z).
A THREAD select after a WARP select binds the lane (0..31); without one it
binds the thread coordinate along its dimension.

An op is a tuple:
  ("group", k, depth)  ("split_fst", k, depth)  ("split_snd", k, depth)
  ("transpose", depth) ("reverse", depth)       ("select", level, dim)
"""
from __future__ import annotations

import numpy as np

GRID, BLOCK, WARP, THREAD = 0, 1, 2, 3
X, Y, Z = 0, 1, 2


class ViewError(ValueError):
    """A view or selection that the view types reject (shape, divisibility,
    select extent vs. resource count, or selection order)."""


def stages(base_shape, ops):
    """Array shape before each op and after the last (list of lists).

    Applies the type of each basic view (listing of basic view types).  A
    select removes the outermost dimension.
    """
    cur = [int(s) for s in base_shape]
    out = []
    for op in ops:
        out.append(list(cur))
        kind = op[0]
        if kind == "select":
            if not cur:
                raise ViewError("select from a scalar")
            cur = cur[1:]
            continue
        d = op[-1]
        if d < 0 or d >= len(cur):
            raise ViewError(f"{kind} at depth {d} of a rank-{len(cur)} array")
        n = cur[d]
        if kind == "group":
            k = op[1]
            if k < 1 or n % k != 0:
                raise ViewError(f"group<{k}> of extent {n}")
            cur = cur[:d] + [n // k, k] + cur[d + 1:]
        elif kind in ("split_fst", "split_snd"):
            k = op[1]
            if not 0 <= k <= n:
                raise ViewError(f"split at {k} of extent {n}")
            cur[d] = k if kind == "split_fst" else n - k
        elif kind == "transpose":
            if d + 1 >= len(cur):
                raise ViewError("transpose needs a nested array")
            cur[d], cur[d + 1] = cur[d + 1], cur[d]
        elif kind == "reverse":
            pass
        else:
            raise ViewError(f"unknown view {kind}")
    out.append(list(cur))
    return out


def selects(base_shape, ops):
    """[(level, dim, extent)] of the selects, in the order they appear."""
    st = stages(base_shape, ops)
    return [(op[1], op[2], st[i][0]) for i, op in enumerate(ops) if op[0] == "select"]


def resource_count(level, dim, grid, block, after_warp):
    """Number of sub-resources a select at (level, dim) distributes over."""
    nthreads = block[0] * block[1] * block[2]
    if level == BLOCK:
        return grid[dim]
    if level == WARP:
        if dim != X or nthreads % 32:
            raise ViewError("warp select needs dim X and a multiple of 32 threads")
        return nthreads // 32
    if level == THREAD:
        if after_warp:
            if dim != X:
                raise ViewError("lane select needs dim X")
            return 32
        return block[dim]
    raise ViewError(f"cannot select at level {level}")


def check_selects(base_shape, ops, grid, block):
    """Select extents equal the resource counts (Section 3.2, select), and
    selections narrow from coarse to fine: block before warp before thread,
    each (level, dim) at most once (Section 3.3, narrowing)."""
    seen, last, after_warp = set(), BLOCK, False
    for level, dim, ext in selects(base_shape, ops):
        if level < last:
            raise ViewError("selection does not narrow grid -> block -> warp -> thread")
        if (level, dim) in seen:
            raise ViewError("resource selected twice")
        seen.add((level, dim))
        last = level
        cnt = resource_count(level, dim, grid, block, after_warp)
        if ext != cnt:
            raise ViewError(f"select extent {ext} != {cnt} resources at level {level} dim {dim}")
        if level == WARP:
            after_warp = True


def resolve(base_shape, ops, bound, local):
    """Raw index in the base array (row-major) of one logical point.

    ``bound`` holds the coordinate of each select, in order; ``local`` the
    coordinates of the dimensions left after the last op.  Works elementwise
    on NumPy integer arrays.  Views are undone starting from the last one.
    """
    st = stages(base_shape, ops)
    coords = list(local)
    nsel = sum(1 for op in ops if op[0] == "select")
    for s in range(len(ops) - 1, -1, -1):
        op, before = ops[s], st[s]
        kind = op[0]
        if kind == "select":
            nsel -= 1
            coords = [bound[nsel]] + coords
            continue
        d = op[-1]
        if kind == "group":
            coords = coords[:d] + [coords[d] * op[1] + coords[d + 1]] + coords[d + 2:]
        elif kind == "split_snd":
            coords[d] = coords[d] + op[1]
        elif kind == "transpose":
            coords[d], coords[d + 1] = coords[d + 1], coords[d]
        elif kind == "reverse":
            coords[d] = (before[d] - 1) - coords[d]
        # split_fst keeps the coordinate
    lin = 0
    for c, n in zip(coords, base_shape):
        lin = lin * int(n) + c
    return lin


def domain_shape(base_shape, ops):
    """Extents of the logical domain: the select extents, then the dims left."""
    st = stages(base_shape, ops)
    return [e for (_, _, e) in selects(base_shape, ops)] + st[-1]


def domain_indices(base_shape, ops):
    """Raw index of every logical point, as an int64 array of the domain
    shape, in logical row-major order (selected dims first, in select order)."""
    dom = domain_shape(base_shape, ops)
    nsel = len(selects(base_shape, ops))
    if not dom:
        return np.array(resolve(base_shape, ops, [], []), dtype=np.int64)
    grids = np.indices(dom, dtype=np.int64) if all(dom) else [np.zeros(dom, np.int64)] * len(dom)
    idx = resolve(base_shape, ops, list(grids[:nsel]), list(grids[nsel:]))
    return np.broadcast_to(np.asarray(idx, dtype=np.int64), dom).copy()


# --------------------------------------------------------------------------
# Access-conflict check (Section 3.3 "Narrowing", "Synchronization";
# Section 4, access_safety_check = narrowing + access conflict)
# --------------------------------------------------------------------------

def thread_coords(grid, block):
    """Per thread of the whole grid: dict of exec coordinates (flat arrays)."""
    bz, by, bx = np.meshgrid(np.arange(grid[2]), np.arange(grid[1]), np.arange(grid[0]), indexing="ij")
    tz, ty, tx = np.meshgrid(np.arange(block[2]), np.arange(block[1]), np.arange(block[0]), indexing="ij")
    nb = grid[0] * grid[1] * grid[2]
    nt = block[0] * block[1] * block[2]
    B = {X: np.repeat(bx.ravel(), nt), Y: np.repeat(by.ravel(), nt), Z: np.repeat(bz.ravel(), nt)}
    T = {X: np.tile(tx.ravel(), nb), Y: np.tile(ty.ravel(), nb), Z: np.tile(tz.ravel(), nb)}
    lin_t = T[X] + block[0] * (T[Y] + block[1] * T[Z])
    lin_b = B[X] + grid[0] * (B[Y] + grid[1] * B[Z])
    tid = lin_b * nt + lin_t
    return B, T, lin_t, tid


def view_access(base_shape, ops, grid, block):
    """(tid, element) pairs of a view accessed by every thread of the grid.

    Each thread takes the logical points whose selected coordinates equal its
    own exec coordinates; exec dimensions the view does not select replicate
    the access (every thread along them touches the same elements).
    """
    check_selects(base_shape, ops, grid, block)
    B, T, lin_t, tid = thread_coords(grid, block)
    sels = selects(base_shape, ops)
    bound, after_warp = [], False
    for level, dim, _ in sels:
        if level == BLOCK:
            bound.append(B[dim])
        elif level == WARP:
            bound.append(lin_t // 32)
            after_warp = True
        else:
            bound.append(lin_t % 32 if after_warp else T[dim])
    local = stages(base_shape, ops)[-1]
    nloc = int(np.prod(local)) if local else 1
    lgrid = np.indices(local, dtype=np.int64).reshape(len(local), -1) if local else np.zeros((0, 1), np.int64)
    nthr = tid.size
    b = [np.repeat(c, nloc) for c in bound]
    loc = [np.tile(lgrid[i], nthr) for i in range(len(local))]
    elem = np.asarray(resolve(base_shape, ops, b, loc), dtype=np.int64)
    elem = np.broadcast_to(elem, (nthr * nloc,))
    return np.repeat(tid, nloc), elem


def affine_access(extent, stride, offset, binds, grid, block):
    """(tid, element) pairs of a raw affine index map, for index code that is
    not written with views (e.g. the CUDA transpose of Section 1).

    element = offset + sum_i coord_i * stride_i over the box ``extent``;
    ``binds[i]`` names what coordinate i is: ("block", dim), ("thread", dim),
    ("warp",), ("lane",) or ("local",).
    """
    B, T, lin_t, tid = thread_coords(grid, block)
    loc_dims = [i for i, b in enumerate(binds) if b[0] == "local"]
    loc_ext = [extent[i] for i in loc_dims]
    nloc = int(np.prod(loc_ext)) if loc_ext else 1
    lgrid = np.indices(loc_ext, dtype=np.int64).reshape(len(loc_ext), -1) if loc_ext else np.zeros((0, 1), np.int64)
    nthr = tid.size
    elem = np.full(nthr * nloc, offset, dtype=np.int64)
    valid = np.ones(nthr * nloc, dtype=bool)
    li = 0
    for i, b in enumerate(binds):
        if b[0] == "local":
            c = np.tile(lgrid[li], nthr)
            li += 1
        else:
            if b[0] == "block":
                c0 = B[b[1]]
            elif b[0] == "thread":
                c0 = T[b[1]]
            elif b[0] == "warp":
                c0 = lin_t // 32
            else:
                c0 = lin_t % 32
            c = np.repeat(c0, nloc)
            valid &= c < extent[i]     # resources beyond the extent do not access
        elem = elem + c * stride[i]
    t = np.repeat(tid, nloc)
    return t[valid], elem[valid]


def first_conflict(accesses):
    """Smallest element index with a conflicting access, or None.

    ``accesses`` is a list of (buffer, tids, elems, is_write).  Two accesses
    conflict when they touch the same element of the same buffer from two
    different threads and at least one of them writes (the data-race
    definition of Section 2.2; the narrowing and access-conflict steps of
    access_safety_check, Section 4, for one phase between barriers).
    """
    worst = None
    buffers = sorted({a[0] for a in accesses})
    for buf in buffers:
        wt = [a[1] for a in accesses if a[0] == buf and a[3]]
        we = [a[2] for a in accesses if a[0] == buf and a[3]]
        rt = [a[1] for a in accesses if a[0] == buf and not a[3]]
        re_ = [a[2] for a in accesses if a[0] == buf and not a[3]]
        if not wt:
            continue
        wt, we = np.concatenate(wt), np.concatenate(we)
        pairs = np.unique(np.stack([we, wt], 1), axis=0)
        e, cnt = np.unique(pairs[:, 0], return_counts=True)
        bad = list(e[cnt > 1])
        writer = dict(zip(pairs[:, 0].tolist(), pairs[:, 1].tolist()))
        if rt:
            rt, re_ = np.concatenate(rt), np.concatenate(re_)
            for el, t in zip(re_.tolist(), rt.tolist()):
                w = writer.get(el)
                if w is not None and w != t:
                    bad.append(el)
        if bad:
            m = int(min(bad))
            worst = m if worst is None else min(worst, m)
    return worst


def views_disjoint(accesses, grid, block):
    """accesses: list of (buffer, base_shape, ops, is_write).  Returns the
    first conflicting element or None."""
    acc = []
    for buf, shape, ops, w in accesses:
        t, e = view_access(shape, ops, grid, block)
        acc.append((buf, t, e, w))
    return first_conflict(acc)
