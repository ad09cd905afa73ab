"""Oracle: reduce, inclusive scan, view copy and segmented reduce+scan
(test infrastructure).

Section 5 names four benchmarks -- block-wide parallel reduction, matrix
transposition, scan and matrix multiplication -- without fixing their
operators or types.  Readings used here: the reduction and the scan are sums
(the scan inclusive), over int32 (two's-complement wrap-around, i.e. exact
arithmetic mod 2^32) or FP32.

All three ops here are defined over views (module ``views``).  The logical
domain of a view is its select dimensions (in select order) followed by the
dimensions left after its last op, in row-major order.

  reduce  out[o] = sum of in[index(p)] over the logical points p whose
          selected coordinates at levels <= out_level linearise to o
  scan    within each segment -- the points sharing their selected coordinates
          at levels <= seg_level -- out[index(p)] = sum of in[index(q)] over
          q <= p in logical order
  copy    out[index_out(p)] = in[index_in(p)] for every logical point p
          (the transpose is the copy whose input view is a transpose)

Integers are summed in int64 and wrapped to int32 at the end.  FP32 sums are
exact (math.fsum, correctly rounded to FP64); FP32 prefix sums are FP64
cumulative sums, whose error is below n * 2^-53 * sum|x| (< 3e-8 * sum|x| for
n <= 2^28), far inside the 1e-5 * sum|x| tolerance they are compared with.
"""
from __future__ import annotations

import math

import numpy as np

from . import views as V


def wrap_i32(v):
    """int64 -> int32 two's-complement wrap-around."""
    v = np.asarray(v, dtype=np.int64)
    return (((v + (1 << 31)) & ((1 << 32) - 1)) - (1 << 31)).astype(np.int32)


def _rows(x, base_shape, ops, keep_level):
    """Values of the logical domain as a 2-D array: one row per combination
    of the selected coordinates at levels <= keep_level, the rest of the
    domain (in logical order) along the row.  Returns (values, raw indices)."""
    idx = V.domain_indices(base_shape, ops)
    sels = V.selects(base_shape, ops)
    nkeep = sum(1 for (lvl, _, _) in sels if lvl <= keep_level)
    rows = int(np.prod([e for (_, _, e) in sels[:nkeep]])) if nkeep else 1
    idx = idx.reshape(rows, -1)
    return np.asarray(x).reshape(-1)[idx], idx


def reduce(x, base_shape, ops, out_level, grid=None, block=None):
    """Sum over the view, one output per resource at ``out_level``
    (GRID: one scalar).  int32 input -> int32 output (wrapped); FP32 input
    -> exact sums in FP64.  Also returns sum|x| per output (FP only)."""
    if grid is not None:
        V.check_selects(base_shape, ops, grid, block)
    vals, _ = _rows(x, base_shape, ops, out_level)
    if vals.dtype == np.int32:
        return wrap_i32(vals.astype(np.int64).sum(axis=1)), None
    s = np.array([math.fsum(r) for r in vals.astype(np.float64)])
    a = np.array([math.fsum(np.abs(r)) for r in vals.astype(np.float64)])
    return s, a


def scan(x, out_init, base_shape, ops, seg_level, grid=None, block=None):
    """Inclusive prefix sums over the view, segmented at ``seg_level``.

    Returns (out, prefix_abs): ``out`` is ``out_init`` with every element the
    view reaches replaced by its prefix sum (int32 wrapped, or FP64), and
    ``prefix_abs`` the matching sum_{q<=p} |x_q| (FP only, else None)."""
    if grid is not None:
        V.check_selects(base_shape, ops, grid, block)
    vals, idx = _rows(x, base_shape, ops, seg_level)
    out = np.array(out_init, copy=True).reshape(-1)
    if vals.dtype == np.int32:
        out[idx.reshape(-1)] = wrap_i32(np.cumsum(vals.astype(np.int64), axis=1)).reshape(-1)
        return out.reshape(np.shape(out_init)), None
    out = out.astype(np.float64)
    pa = np.zeros_like(out)
    out[idx.reshape(-1)] = np.cumsum(vals.astype(np.float64), axis=1).reshape(-1)
    pa[idx.reshape(-1)] = np.cumsum(np.abs(vals.astype(np.float64)), axis=1).reshape(-1)
    return out.reshape(np.shape(out_init)), pa.reshape(np.shape(out_init))


def view_copy(x, out_init, in_shape, in_ops, out_shape, out_ops):
    """out[index_out(p)] = in[index_in(p)] over the common logical domain."""
    if V.domain_shape(in_shape, in_ops) != V.domain_shape(out_shape, out_ops):
        raise V.ViewError("input and output views have different domains")
    ii = V.domain_indices(in_shape, in_ops).reshape(-1)
    oi = V.domain_indices(out_shape, out_ops).reshape(-1)
    out = np.array(out_init, copy=True).reshape(-1)
    out[oi] = np.asarray(x).reshape(-1)[ii]
    return out.reshape(np.shape(out_init))


def transpose2d(x):
    """out[j][i] = in[i][j] for a row-major R x C matrix, element by element."""
    R, C = x.shape
    out = np.empty((C, R), dtype=x.dtype)
    for i in range(R):
        out[:, i] = x[i, :]
    return out


def segmented_reduce_scan(x, offsets):
    """Per segment s = [offsets[s], offsets[s+1]): its sum and its inclusive
    prefix sums.  Returns (scan (FP64 / wrapped int32), sums, prefix |x|,
    sum |x| per segment).  Empty segments have sum 0."""
    x = np.asarray(x)
    off = np.asarray(offsets, dtype=np.int64)
    S = off.size - 1
    is_int = x.dtype == np.int32
    scan_out = np.zeros(x.size, dtype=np.int32 if is_int else np.float64)
    pa = None if is_int else np.zeros(x.size, dtype=np.float64)
    sums = np.zeros(S, dtype=np.int32 if is_int else np.float64)
    sabs = None if is_int else np.zeros(S, dtype=np.float64)
    for s in range(S):
        a, b = int(off[s]), int(off[s + 1])
        seg = x[a:b]
        if is_int:
            scan_out[a:b] = wrap_i32(np.cumsum(seg.astype(np.int64)))
            sums[s] = wrap_i32(seg.astype(np.int64).sum())
        else:
            seg64 = seg.astype(np.float64)
            scan_out[a:b] = np.cumsum(seg64)
            pa[a:b] = np.cumsum(np.abs(seg64))
            sums[s] = math.fsum(seg64)
            sabs[s] = math.fsum(np.abs(seg64))
    return scan_out, sums, pa, sabs


# ---- other operators ----------------------------------------------------------
# Section 5 fixes no operator for its reduction and scan; a generic reduce or
# scan takes any associative operator.  Besides the sum:
#   max / min    exact; on FP32 they follow IEEE maxNum / minNum, so a NaN
#                operand is ignored unless every operand is NaN
#   prod         int32: the product modulo 2^32 (exact integers, wrapped);
#                FP32: the FP64 product of the FP32 inputs (relative error at
#                most (m - 1) 2^-53 for m factors, far inside the FP32 bound
#                it is compared with)
#   and/or/xor   int32 bitwise
#   argmax/argmin  the index in the base array of the element holding the
#                largest / smallest value; among equal values the smallest
#                index; FP32 NaNs lose to every number (all NaN: the smallest
#                index); -1 for no element
# and exclusive scans, where a point gets the combination of the points
# strictly before it in its segment (the operator's identity for the first).

OPS = ("sum", "max", "min", "prod", "and", "or", "xor", "argmax", "argmin")


def identity(op, is_int):
    """The value of an empty reduction under op."""
    if op in ("sum", "or", "xor"):
        return 0
    if op == "max":
        return np.iinfo(np.int32).min if is_int else -np.inf
    if op == "min":
        return np.iinfo(np.int32).max if is_int else np.inf
    if op == "prod":
        return 1
    if op == "and":
        return -1
    return -1                                            # argmax / argmin: no element


def arg_pick(vals, idx, op):
    """The arg-maximum / arg-minimum of one set of (value, element index)
    pairs, from the definition: the best value among the non-NaN ones (all
    NaN: every element ties), then the smallest index holding it."""
    vals = np.asarray(vals, dtype=np.float64)
    idx = np.asarray(idx, dtype=np.int64)
    if vals.size == 0:
        return -1
    num = ~np.isnan(vals)
    if not num.any():
        return int(idx.min())
    best = vals[num].max() if op == "argmax" else vals[num].min()
    return int(idx[num & (vals == best)].min())


def _arg_prefix(vals, idx, op, exclusive):
    """Running arg operator along one row, point by point in logical order."""
    out = np.empty(vals.size, dtype=np.int64)
    bv, bi = None, -1
    for p in range(vals.size):
        if exclusive:
            out[p] = bi
        v, i = float(vals[p]), int(idx[p])
        if bi < 0:
            take = True
        elif np.isnan(v) != np.isnan(bv):
            take = not np.isnan(v)
        elif np.isnan(v):
            take = i < bi
        elif v != bv:
            take = v > bv if op == "argmax" else v < bv
        else:
            take = i < bi
        if take:
            bv, bi = v, i
        if not exclusive:
            out[p] = bi
    return out


def _wrap_prod_prefix(row):
    """Prefix products of int32 values modulo 2^32 (exact Python integers)."""
    out, acc = [], 1
    for v in row.tolist():
        acc = (acc * int(v)) & 0xFFFFFFFF
        out.append(acc)
    return wrap_i32(np.array(out, dtype=np.int64) - ((np.array(out, dtype=np.int64) >> 31) << 32))


def _combine_rows(vals, op, exclusive, idx=None):
    """Prefix combination along each row (inclusive or exclusive): sums in
    int64 (wrapped later) or FP64, max / min / bitwise exactly, int32
    products exactly modulo 2^32, FP32 products in FP64, arg operators as
    element indices (``idx``: the base-array index of every value)."""
    is_int = vals.dtype == np.int32
    if op in ("argmax", "argmin"):
        return np.array([_arg_prefix(vals[r], idx[r], op, exclusive) for r in range(vals.shape[0])],
                        dtype=np.int64).reshape(vals.shape)
    if op == "sum":
        v = vals.astype(np.int64 if is_int else np.float64)
        inc = np.cumsum(v, axis=1)
    elif op == "prod" and is_int:
        inc = np.array([_wrap_prod_prefix(r) for r in vals], dtype=np.int64).reshape(vals.shape)
    elif op == "prod":
        inc = np.multiply.accumulate(vals.astype(np.float64), axis=1) if vals.shape[1] else vals.astype(np.float64)
    elif op in ("and", "or", "xor"):
        f = {"and": np.bitwise_and, "or": np.bitwise_or, "xor": np.bitwise_xor}[op]
        inc = f.accumulate(vals.astype(np.int64), axis=1) if vals.shape[1] else vals.astype(np.int64)
    else:
        f = np.fmax if op == "max" else np.fmin
        v = vals.astype(np.int64 if is_int else np.float64)
        inc = f.accumulate(v, axis=1) if v.shape[1] else v
    if not exclusive:
        return inc
    out = np.empty_like(inc)
    if inc.shape[1]:
        out[:, 0] = identity(op, is_int)
        out[:, 1:] = inc[:, :-1]
    return out


def _reduce_row(r, ri, op, is_int):
    """One output of reduce_op: the plain definition of each operator."""
    if r.size == 0:
        return identity(op, is_int)
    if op == "sum":
        return int(wrap_i32(r.astype(np.int64).sum())) if is_int else math.fsum(r.astype(np.float64))
    if op in ("argmax", "argmin"):
        return arg_pick(r, ri, op)
    if op == "prod" and is_int:
        acc = 1
        for v in r.tolist():
            acc = (acc * int(v)) & 0xFFFFFFFF
        return acc - (1 << 32) if acc >= (1 << 31) else acc
    if op == "prod":
        return float(np.prod(r.astype(np.float64)))
    if op in ("and", "or", "xor"):
        f = {"and": np.bitwise_and, "or": np.bitwise_or, "xor": np.bitwise_xor}[op]
        return int(f.reduce(r.astype(np.int64)))
    f = np.fmax if op == "max" else np.fmin
    return f.reduce(r)


def reduce_op(x, base_shape, ops, out_level, op, grid=None, block=None):
    """The reduction under op (see OPS) over the view, one output per
    resource at ``out_level``; the identity for an empty row.  int32
    results (all arg operators, int32 inputs) as int32, FP32 ones in FP64."""
    if grid is not None:
        V.check_selects(base_shape, ops, grid, block)
    vals, idx = _rows(x, base_shape, ops, out_level)
    is_int = vals.dtype == np.int32
    out = [_reduce_row(r, ri, op, is_int) for r, ri in zip(vals, idx)]
    if is_int or op in ("argmax", "argmin"):
        return np.array(out, dtype=np.int64).astype(np.int32)
    return np.array(out, dtype=np.float64)


def scan_op(x, out_init, base_shape, ops, seg_level, op="sum", exclusive=False, grid=None, block=None):
    """Prefix combination over the view, segmented at ``seg_level``, with an
    operator of OPS, inclusive or exclusive.  Returns (out, prefix_abs):
    prefix_abs is sum |x| over the combined points (FP sums only, else
    None), the scale of the sum's tolerance.  Arg operators write int32
    element indices (out_init should then be int32)."""
    if grid is not None:
        V.check_selects(base_shape, ops, grid, block)
    vals, idx = _rows(x, base_shape, ops, seg_level)
    is_int = vals.dtype == np.int32
    res = _combine_rows(vals, op, exclusive, idx)
    out = np.array(out_init, copy=True).reshape(-1)
    if op in ("argmax", "argmin"):
        out = out.astype(np.int32)
        out[idx.reshape(-1)] = res.astype(np.int32).reshape(-1)
        return out.reshape(np.shape(out_init)), None
    if is_int:
        out[idx.reshape(-1)] = wrap_i32(res).reshape(-1) if op in ("sum", "prod") else \
            res.astype(np.int32).reshape(-1)
        return out.reshape(np.shape(out_init)), None
    out = out.astype(np.float64)
    out[idx.reshape(-1)] = res.reshape(-1)
    pa = None
    if op == "sum":
        pa = np.zeros_like(out)
        pa[idx.reshape(-1)] = _combine_rows(np.abs(vals.astype(np.float64)).astype(np.float32), "sum",
                                            exclusive).reshape(-1)
    return out.reshape(np.shape(out_init)), pa if pa is None else pa.reshape(np.shape(out_init))


def segmented_op(x, offsets, op="sum", exclusive=False):
    """Per segment [offsets[s], offsets[s+1]): the prefix combination
    (inclusive or exclusive) and the total, under op.  Returns (scan, totals,
    prefix |x| (FP sums), total |x| (FP sums)); empty segments total the
    identity.  Arg operators give int32 indices into x."""
    x = np.asarray(x)
    off = np.asarray(offsets, dtype=np.int64)
    S = off.size - 1
    is_int = x.dtype == np.int32
    arg = op in ("argmax", "argmin")
    as_int = is_int or arg
    scan_out = np.zeros(x.size, dtype=np.int32 if as_int else np.float64)
    tot = np.zeros(S, dtype=np.int32 if as_int else np.float64)
    fp_sum = (not is_int) and op == "sum"
    pa = np.zeros(x.size) if fp_sum else None
    sabs = np.zeros(S) if fp_sum else None
    for s in range(S):
        a, b = int(off[s]), int(off[s + 1])
        seg = x[a:b].reshape(1, -1)
        sidx = np.arange(a, b, dtype=np.int64).reshape(1, -1)
        r = _combine_rows(seg, op, exclusive, sidx).reshape(-1)
        if arg:
            scan_out[a:b] = r
            tot[s] = arg_pick(seg.reshape(-1), sidx.reshape(-1), op)
        elif is_int:
            scan_out[a:b] = wrap_i32(r) if op in ("sum", "prod") else r.astype(np.int32)
            t = _reduce_row(seg.reshape(-1), sidx.reshape(-1), op, True)
            tot[s] = wrap_i32(t) if op == "sum" else np.int32(t)
        else:
            scan_out[a:b] = r
            tot[s] = (math.fsum(seg.reshape(-1).astype(np.float64)) if op == "sum" else
                      _reduce_row(seg.reshape(-1), sidx.reshape(-1), op, False)) if b > a else identity(op, False)
            if fp_sum:
                pa[a:b] = _combine_rows(np.abs(seg).astype(np.float32), "sum", exclusive).reshape(-1)
                sabs[s] = math.fsum(np.abs(seg.reshape(-1).astype(np.float64)))
    return scan_out, tot, pa, sabs


def prod_tolerance(m):
    """gamma_(m-1) = (m - 1) u / (1 - (m - 1) u), u = 2^-24: the relative error
    bound of a product of m FP32 factors computed in FP32 in any order (no
    overflow or underflow), each multiplication rounding to nearest."""
    k = max(int(m) - 1, 0) * 2.0 ** -24
    return k / (1.0 - k)
