"""Python binding of libdesc (argument marshalling only).

Every operation runs in libdesc.so's own CUDA kernels for sm_103a; this
module only converts view descriptions and torch tensors into the C ABI of
``include/desc.h`` and raises ``DescError`` on a non-OK status.  torch
supplies device memory and streams.  There is no fallback: if libdesc.so has
not been built, importing the library raises.

Views are written as tuples, ops applied left to right:
  ("group", k, depth) ("split_fst", k, depth) ("split_snd", k, depth)
  ("transpose", depth) ("reverse", depth) ("select", level, dim)
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_int32, c_int64, c_size_t, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdesc.so")

GRID, BLOCK, WARP, THREAD = 0, 1, 2, 3
X, Y, Z, LANE = 0, 1, 2, 3
I32, F32 = 0, 1
MM_FP32_SIMT, MM_BF16, MM_SPLIT3, MM_SPLIT2 = 0, 1, 2, 3
OP_REDUCE, OP_SCAN, OP_TRANSPOSE, OP_SEGMENTED, OP_MATMUL = 0, 1, 2, 3, 4
NUM_FEATURES = 40
KAHAN = 1
MAX, MIN, EXCLUSIVE = 1 << 1, 1 << 2, 1 << 3
PROD, AND, OR, XOR, ARGMAX, ARGMIN = 1 << 4, 1 << 5, 1 << 6, 1 << 7, 1 << 8, 1 << 9
ARG_FLAGS = ARGMAX | ARGMIN
DEBUG_STALL_TILE = 1 << 16
CHECK_OFFSETS = 1 << 17

STATUS = {0: "DESC_OK", 1: "DESC_ERR_INVALID_ARG", 2: "DESC_ERR_SHAPE", 3: "DESC_ERR_OVERLAP",
          4: "DESC_ERR_HOST_POINTER", 5: "DESC_ERR_SIZE_MISMATCH", 6: "DESC_ERR_ALIGNMENT",
          7: "DESC_ERR_UNSUPPORTED", 8: "DESC_ERR_CUDA", 9: "DESC_ERR_DEVICE_TIMEOUT",
          10: "DESC_ERR_WORKSPACE"}
_KIND = {"group": 0, "split_fst": 1, "split_snd": 2, "transpose": 3, "reverse": 4, "select": 5}
MAX_RANK, MAX_OPS, MAX_DIMS = 4, 16, 20


class DescError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


class ViewOp(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("depth", c_int32), ("k", c_int64), ("level", c_int32), ("dim", c_int32)]


class View(ctypes.Structure):
    _fields_ = [("rank", c_int32), ("nops", c_int32), ("shape", c_int64 * MAX_RANK), ("ops", ViewOp * MAX_OPS)]


class Exec(ctypes.Structure):
    _fields_ = [("grid", c_int64 * 3), ("block", c_int64 * 3)]


class Lowered(ctypes.Structure):
    _fields_ = [("ndims", c_int32), ("nsel", c_int32), ("extent", c_int64 * MAX_DIMS),
                ("stride", c_int64 * MAX_DIMS), ("level", c_int32 * MAX_DIMS), ("dim", c_int32 * MAX_DIMS),
                ("offset", c_int64), ("base_elems", c_int64)]

    def as_dict(self):
        n = self.ndims
        return {"ndims": n, "nsel": self.nsel, "extent": list(self.extent[:n]), "stride": list(self.stride[:n]),
                "level": list(self.level[:n]), "dim": list(self.dim[:n]), "offset": self.offset,
                "base_elems": self.base_elems}


class Access(ctypes.Structure):
    _fields_ = [("map", Lowered), ("buffer", c_int32), ("is_write", c_int32)]


class Stmt(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("level", c_int32), ("dim", c_int32), ("n_first", c_int32),
                ("n_second", c_int32), ("at", c_int64), ("access", Access)]


class Problem(ctypes.Structure):
    _fields_ = [("op", c_int32), ("dtype", c_int32), ("n", c_int64), ("aux", c_int64), ("k", c_int64),
                ("seg_lengths", POINTER(c_int64)), ("view", POINTER(View)), ("ex", POINTER(Exec)),
                ("level", c_int32)]


class MmPlan(ctypes.Structure):
    _fields_ = [("candidate", c_int32), ("pairs", c_int32), ("tile_n", c_int32), ("padded", c_int32),
                ("rows", c_int64), ("tiles", c_int64), ("whole_tiles", c_int64), ("pieces", c_int32),
                ("max_pairs", c_int32)]


class TuneBuffers(ctypes.Structure):
    _fields_ = [("inp", c_void_p), ("out", c_void_p), ("sums", c_void_p), ("offsets", c_void_p), ("ws", c_void_p),
                ("ws_bytes", c_size_t), ("in2", c_void_p)]


_lib_handle = None


def lib():
    """The loaded libdesc.so (raises if it has not been built)."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        _declare(L)
        _lib_handle = L
    return _lib_handle


def _declare(L):
    P = c_void_p
    sig = {
        "desc_status_string": (c_char_p, [c_int32]),
        "desc_version": (c_int32, []),
        "desc_lower_view": (c_int32, [POINTER(View), POINTER(Exec), POINTER(Lowered)]),
        "desc_check_disjoint": (c_int32, [POINTER(Access), c_int32, POINTER(Exec), POINTER(c_int64)]),
        "desc_check_disjoint_ex": (c_int32, [POINTER(Access), c_int32, POINTER(Exec), POINTER(c_int64),
                                             POINTER(c_int32)]),
        "desc_check_program": (c_int32, [POINTER(Stmt), c_int32, POINTER(Exec), POINTER(c_int32), POINTER(c_int64)]),
        "desc_split_reduce_transpose": (c_int32, [POINTER(View), POINTER(Exec), c_int32, c_int32, c_void_p, c_size_t,
                                                  c_void_p, c_size_t, c_void_p, c_size_t, c_void_p, c_void_p, c_int64,
                                                  c_int64, c_void_p]),
        "desc_reduce_workspace_size": (c_int32, [POINTER(View), POINTER(Exec), c_int32, c_int32, POINTER(c_size_t)]),
        "desc_reduce": (c_int32, [POINTER(View), POINTER(Exec), c_int32, c_int32, P, c_size_t, P, c_size_t,
                                  c_int32, P, c_size_t, P]),
        "desc_scan_workspace_size": (c_int32, [POINTER(View), POINTER(Exec), c_int32, c_int32, POINTER(c_size_t)]),
        "desc_scan": (c_int32, [POINTER(View), POINTER(Exec), c_int32, c_int32, P, c_size_t, P, c_size_t,
                                c_int32, P, c_size_t, P]),
        "desc_transpose": (c_int32, [POINTER(View), POINTER(View), POINTER(Exec), c_int32, P, c_size_t, P,
                                     c_size_t, P]),
        "desc_stream_status": (c_int32, [P]),
        "desc_matmul_workspace_size": (c_int32, [c_int64, c_int64, c_int64, c_int32, POINTER(c_size_t)]),
        "desc_matmul_plan": (c_int32, [c_int64, c_int64, c_int64, c_int32, c_int32, c_int32, POINTER(MmPlan)]),
        "desc_matmul": (c_int32, [POINTER(View), POINTER(View), c_int64, c_int64, c_int64, P, c_size_t, P, c_size_t,
                                  P, c_size_t, c_int32, P, c_size_t, P]),
        "desc_segmented_workspace_size": (c_int32, [c_int64, c_int64, POINTER(c_size_t)]),
        "desc_segmented_reduce_scan": (c_int32, [P, c_int64, c_int64, c_int32, P, P, P, c_int32, P, c_size_t, P]),
        "desc_segmented_graph_create": (c_int32, [P, c_int64, c_int64, c_int32, P, P, P, P, c_size_t,
                                                  POINTER(c_void_p)]),
        "desc_graph_launch": (c_int32, [c_void_p, P]),
        "desc_graph_destroy": (c_int32, [c_void_p]),
        "desc_segmented_reduce_scan_per_segment": (c_int32, [POINTER(c_int64), c_int64, c_int32, P, P, P, P,
                                                             c_size_t, P]),
        "desc_candidate_count": (c_int32, [c_int32, POINTER(c_int32)]),
        "desc_features": (c_int32, [POINTER(Problem), c_int32, POINTER(ctypes.c_float), c_int32]),
        "desc_tune_measure": (c_int32, [POINTER(Problem), POINTER(TuneBuffers), c_int32, P, POINTER(ctypes.c_float)]),
        "desc_tune_measure_cands": (c_int32, [POINTER(Problem), POINTER(TuneBuffers), POINTER(c_int32), c_int32,
                                              c_int32, P, POINTER(ctypes.c_float)]),
        "desc_tune_exhaustive": (c_int32, [POINTER(Problem), POINTER(TuneBuffers), c_int32, P, POINTER(c_int32)]),
        "desc_tune_record": (c_int32, [POINTER(Problem), c_int32]),
        "desc_tune_lookup": (c_int32, [POINTER(Problem), POINTER(c_int32)]),
        "desc_tune_clear": (c_int32, []),
        "desc_tune_save": (c_int32, [c_char_p]),
        "desc_tune_load": (c_int32, [c_char_p]),
        "desc_force_candidate": (c_int32, [c_int32, c_int32]),
        "desc_force_generic": (c_int32, [c_int32]),
        "desc_mlp_param_count": (c_int32, [c_int32, c_int32, POINTER(c_int64)]),
        "desc_mlp_workspace_size": (c_int32, [c_int32, c_int32, c_int64, POINTER(c_size_t)]),
        "desc_mlp_forward": (c_int32, [P, c_int32, c_int32, P, c_int64, P, P, c_size_t, P]),
        "desc_mlp_backward": (c_int32, [P, c_int32, c_int32, P, P, c_int64, P, P, c_size_t, P]),
        "desc_mlp_adam": (c_int32, [P, P, P, P, c_int64, c_int32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, P]),
        "desc_mlp_train": (c_int32, [P, P, P, P, c_int32, c_int32, P, P, c_int64, c_int32, c_int32, ctypes.c_float,
                                     P, c_size_t, P, POINTER(ctypes.c_float)]),
        "desc_mlp_pick": (c_int32, [P, c_int32, c_int32, P, c_int32, P, P, P]),
        "desc_tune_set_model": (c_int32, [P, c_int32, c_int32]),
        "desc_tune_predict": (c_int32, [POINTER(Problem), P, POINTER(c_int32)]),
        "desc_scan_noalloc": (c_int32, [POINTER(View), POINTER(Exec), c_int32, c_int32, P, c_size_t, P, c_size_t,
                                        P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


# ----------------------------------------------------------------- marshalling
def make_view(base_shape, ops) -> View:
    v = View()
    if not 1 <= len(base_shape) <= MAX_RANK or len(ops) > MAX_OPS:
        raise DescError(2, "view rank or op count")
    v.rank = len(base_shape)
    v.nops = len(ops)
    for i, s in enumerate(base_shape):
        v.shape[i] = int(s)
    for i, op in enumerate(ops):
        o = v.ops[i]
        o.kind = _KIND[op[0]]
        if op[0] == "select":
            o.level, o.dim, o.depth, o.k = int(op[1]), int(op[2]), 0, 0
        elif op[0] in ("transpose", "reverse"):
            o.depth, o.k = int(op[1]), 0
        else:
            o.k, o.depth = int(op[1]), int(op[2])
    return v


def make_exec(grid=None, block=None):
    if grid is None:
        return None
    e = Exec()
    for i in range(3):
        e.grid[i] = int(grid[i])
        e.block[i] = int(block[i])
    return e


def _ref(x):
    return ctypes.byref(x) if x is not None else None


def _check(st, what):
    if st != 0:
        raise DescError(st, what)


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


def _dtype_code(t):
    import torch
    if t.dtype == torch.int32:
        return I32
    if t.dtype == torch.float32:
        return F32
    raise DescError(1, f"dtype {t.dtype}")


def _ptr(t):
    return c_void_p(t.data_ptr()) if t.numel() else c_void_p(0)


# ----------------------------------------------------------------- host-only ops
def desc_lower_view(base_shape, ops, grid=None, block=None) -> dict:
    out = Lowered()
    _check(lib().desc_lower_view(ctypes.byref(make_view(base_shape, ops)), _ref(make_exec(grid, block)),
                                 ctypes.byref(out)), "desc_lower_view")
    return out.as_dict()


def lowered_struct(d: dict) -> Lowered:
    m = Lowered()
    m.ndims, m.nsel = d["ndims"], d["nsel"]
    for i in range(d["ndims"]):
        m.extent[i], m.stride[i] = d["extent"][i], d["stride"][i]
        m.level[i], m.dim[i] = d["level"][i], d["dim"][i]
    m.offset = d["offset"]
    m.base_elems = d.get("base_elems", 0)
    return m


DECIDED_STRUCTURAL, DECIDED_ENUMERATION = 1, 2


def desc_check_disjoint(accesses, grid, block, with_method=False):
    """accesses: list of (lowered dict, buffer id, is_write).  Returns None
    when the accesses are disjoint, else the first conflicting element; with
    with_method, (that, the DECIDED_* bits of the checks that decided)."""
    n = len(accesses)
    arr = (Access * max(n, 1))()
    for i, (m, buf, w) in enumerate(accesses):
        arr[i].map = lowered_struct(m)
        arr[i].buffer = int(buf)
        arr[i].is_write = 1 if w else 0
    first, how = c_int64(-1), c_int32(0)
    st = lib().desc_check_disjoint_ex(arr, n, ctypes.byref(make_exec(grid, block)), ctypes.byref(first),
                                      ctypes.byref(how))
    if st == 3:
        res = first.value
    else:
        _check(st, "desc_check_disjoint")
        res = None
    return (res, how.value) if with_method else res


STMT_ACCESS, STMT_SYNC, STMT_SPLIT = 0, 1, 2


def _flatten_program(prog, out):
    """Nested statements -> flat Stmt list (preorder); returns the count."""
    start = len(out)
    for st in prog:
        kind = st[0]
        if kind == "access":
            _, buf, base_shape, ops, w = st
            x = Stmt()
            x.kind = STMT_ACCESS
            x.access.map = lowered_struct(desc_lower_view(base_shape, ops))
            x.access.buffer = int(buf)
            x.access.is_write = 1 if w else 0
            out.append(x)
        elif kind == "sync":
            x = Stmt()
            x.kind, x.level = STMT_SYNC, int(st[1])
            out.append(x)
        elif kind == "split":
            _, level, dim, at, first, second = st
            x = Stmt()
            x.kind, x.level, x.dim, x.at = STMT_SPLIT, int(level), int(dim), int(at)
            out.append(x)
            x.n_first = _flatten_program(first, out)
            x.n_second = _flatten_program(second, out)
        else:
            raise DescError(1, f"statement {kind!r}")
    return len(out) - start


def desc_check_program(prog, grid, block):
    """Access safety of a kernel body.  ``prog`` is a list of statements:
    ("access", buffer, base_shape, ops, is_write), ("sync", level) and
    ("split", level, dim, at, [first part], [second part]).  Views are
    lowered without a resource (their select extents are checked against
    the sub-resource by the checker).  Returns (status, statement index,
    first conflicting element): status 0 (safe), 3 (DESC_ERR_OVERLAP),
    11 (DESC_ERR_BARRIER) or 2 (DESC_ERR_SHAPE); statement indices count the
    flattened preorder.  Other statuses raise DescError."""
    flat = []
    _flatten_program(prog, flat)
    arr = (Stmt * max(len(flat), 1))(*flat)
    bad, first = c_int32(-1), c_int64(-1)
    st = lib().desc_check_program(arr, len(flat), ctypes.byref(make_exec(grid, block)), ctypes.byref(bad),
                                  ctypes.byref(first))
    if st not in (0, 2, 3, 11):
        _check(st, "desc_check_program")
    return st, bad.value, (first.value if st == 3 else None)


# ----------------------------------------------------------------- device ops
def _workspace(nbytes, device):
    import torch
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def desc_reduce(x, base_shape, ops, out_level, grid=None, block=None, kahan=False, out=None,
                ws=None, stream=None, flags=0):
    """Sum of tensor ``x`` (the base array) through a view; returns ``out``.
    flags: one operator flag (MAX, MIN, PROD, AND, OR, XOR, ARGMAX, ARGMIN)
    for that operator instead; the arg operators give int32 element indices."""
    import torch
    L = lib()
    v, e = make_view(base_shape, ops), make_exec(grid, block)
    dt = _dtype_code(x)
    if out is None:
        low = desc_lower_view(base_shape, ops, grid, block)
        nout = 1
        for i in range(low["nsel"]):
            if low["level"][i] <= out_level:
                nout *= low["extent"][i]
        out = torch.empty(nout, dtype=torch.int32 if flags & ARG_FLAGS else x.dtype, device=x.device)
    if ws is None:
        nb = c_size_t(0)
        _check(L.desc_reduce_workspace_size(ctypes.byref(v), _ref(e), out_level, dt, ctypes.byref(nb)),
               "desc_reduce_workspace_size")
        ws = _workspace(nb.value, x.device)
    _check(L.desc_reduce(ctypes.byref(v), _ref(e), out_level, dt, _ptr(x), x.numel() * 4, _ptr(out),
                         out.numel() * 4, (KAHAN if kahan else 0) | flags, _ptr(ws), ws.numel(), _stream(stream)),
           "desc_reduce")
    return out


def desc_scan(x, base_shape, ops, seg_level, grid=None, block=None, out=None, ws=None, flags=0,
              stream=None):
    """Inclusive scan of ``x`` through a view into ``out`` (same base array);
    flags as desc_reduce, plus EXCLUSIVE (arg operators: int32 indices)."""
    import torch
    L = lib()
    v, e = make_view(base_shape, ops), make_exec(grid, block)
    dt = _dtype_code(x)
    if out is None:
        out = torch.empty_like(x, dtype=torch.int32) if flags & ARG_FLAGS else torch.empty_like(x)
    if ws is None:
        nb = c_size_t(0)
        _check(L.desc_scan_workspace_size(ctypes.byref(v), _ref(e), seg_level, dt, ctypes.byref(nb)),
               "desc_scan_workspace_size")
        ws = _workspace(nb.value, x.device)
    _check(L.desc_scan(ctypes.byref(v), _ref(e), seg_level, dt, _ptr(x), x.numel() * 4, _ptr(out),
                       out.numel() * 4, flags, _ptr(ws), ws.numel(), _stream(stream)), "desc_scan")
    return out


def desc_split_reduce_transpose(x, base_shape, ops, out_level, grid, block, t_in, t_out, out=None, ws=None,
                                stream=None):
    """One launch: the sum of x through a view (as desc_reduce) on the first
    blocks, t_out = t_in^T (2-D FP32) on the others.  Returns ``out``."""
    import torch
    L = lib()
    v, e = make_view(base_shape, ops), make_exec(grid, block)
    if out is None:
        low = desc_lower_view(base_shape, ops, grid, block)
        nout = 1
        for i in range(low["nsel"]):
            if low["level"][i] <= out_level:
                nout *= low["extent"][i]
        out = torch.empty(nout, dtype=x.dtype, device=x.device)
    if ws is None:
        nb = c_size_t(0)
        _check(L.desc_reduce_workspace_size(ctypes.byref(v), _ref(e), out_level, _dtype_code(x), ctypes.byref(nb)),
               "desc_reduce_workspace_size")
        ws = _workspace(nb.value, x.device)
    R, C = t_in.shape
    _check(L.desc_split_reduce_transpose(ctypes.byref(v), _ref(e), out_level, _dtype_code(x), _ptr(x), x.numel() * 4,
                                         _ptr(out), out.numel() * 4, _ptr(ws), ws.numel(), _ptr(t_in), _ptr(t_out),
                                         int(R), int(C), _stream(stream)), "desc_split_reduce_transpose")
    return out


def desc_transpose(x, in_shape, in_ops, out, out_shape, out_ops, grid=None, block=None, stream=None):
    """out[index_out(p)] = x[index_in(p)] over the common logical domain."""
    _check(lib().desc_transpose(ctypes.byref(make_view(in_shape, in_ops)), ctypes.byref(make_view(out_shape, out_ops)),
                                _ref(make_exec(grid, block)), _dtype_code(x), _ptr(x), x.numel() * 4, _ptr(out),
                                out.numel() * 4, _stream(stream)), "desc_transpose")
    return out


def desc_matmul(A, B, precision, a_view=None, b_view=None, M=None, N=None, K=None, out=None, ws=None,
                stream=None):
    """C = A B (FP32).  A and B are device tensors; by default row-major
    (M x K) and (K x N).  a_view / b_view: (base_shape, ops) views of the
    buffers (lowering to 2-D maps), e.g. a transposed operand."""
    import torch
    L = lib()
    if M is None:
        M = A.shape[0] if a_view is None else None
    if a_view is not None or b_view is not None:
        if M is None or N is None or K is None:
            raise DescError(1, "desc_matmul: M, N, K are needed with views")
    else:
        M, K = A.shape
        N = B.shape[1]
    av = make_view(*a_view) if a_view is not None else None
    bv = make_view(*b_view) if b_view is not None else None
    if out is None:
        out = torch.empty(M, N, dtype=torch.float32, device=A.device)
    if ws is None:
        nb = c_size_t(0)
        _check(L.desc_matmul_workspace_size(M, N, K, precision, ctypes.byref(nb)), "desc_matmul_workspace_size")
        ws = _workspace(nb.value, A.device)
    _check(L.desc_matmul(_ref(av), _ref(bv), M, N, K, _ptr(A), A.numel() * 4, _ptr(B), B.numel() * 4, _ptr(out),
                         out.numel() * 4, precision, _ptr(ws), ws.numel(), _stream(stream)), "desc_matmul")
    return out


def desc_matmul_plan(M, N, K, precision, candidate=-1, max_pairs=0) -> dict:
    """The schedule a tensor-core desc_matmul takes for this shape (no
    launch): candidate -1 is what desc_matmul would take; max_pairs 0 asks
    the current device."""
    pl = MmPlan()
    _check(lib().desc_matmul_plan(M, N, K, precision, candidate, max_pairs, ctypes.byref(pl)), "desc_matmul_plan")
    return {name: getattr(pl, name) for name, _ in MmPlan._fields_}


def desc_segmented_workspace(nseg, total, device):
    nb = c_size_t(0)
    _check(lib().desc_segmented_workspace_size(nseg, total, ctypes.byref(nb)), "desc_segmented_workspace_size")
    return _workspace(nb.value, device)


def desc_segmented_reduce_scan(x, offsets, out=None, sums=None, ws=None, flags=0, stream=None):
    """Per-segment inclusive scans and totals of x (segments from the device
    int64 CSR offsets) in one launch.  Returns (out, sums)."""
    import torch
    nseg = offsets.numel() - 1
    odt = torch.int32 if flags & ARG_FLAGS else x.dtype
    if out is None:
        out = torch.empty_like(x, dtype=odt)
    if sums is None:
        sums = torch.empty(nseg, dtype=odt, device=x.device)
    if ws is None:
        ws = desc_segmented_workspace(nseg, x.numel(), x.device)
    _check(lib().desc_segmented_reduce_scan(_ptr(offsets), nseg, x.numel(), _dtype_code(x), _ptr(x), _ptr(out),
                                            _ptr(sums), flags, _ptr(ws), ws.numel(), _stream(stream)),
           "desc_segmented_reduce_scan")
    return out, sums


class SegmentedGraph:
    """desc_segmented_reduce_scan captured once as a CUDA graph and replayed."""

    def __init__(self, x, offsets, out, sums, ws=None):
        self.keep = (x, offsets, out, sums)
        self.ws = ws if ws is not None else desc_segmented_workspace(offsets.numel() - 1, x.numel(), x.device)
        h = c_void_p(0)
        _check(lib().desc_segmented_graph_create(_ptr(offsets), offsets.numel() - 1, x.numel(), _dtype_code(x),
                                                 _ptr(x), _ptr(out), _ptr(sums), _ptr(self.ws), self.ws.numel(),
                                                 ctypes.byref(h)), "desc_segmented_graph_create")
        self.handle = h

    def launch(self, stream=None):
        _check(lib().desc_graph_launch(self.handle, _stream(stream)), "desc_graph_launch")

    def close(self):
        if self.handle:
            lib().desc_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def desc_segmented_reduce_scan_per_segment(x, h_offsets, out=None, sums=None, ws=None, stream=None):
    """Baseline: one scan and one reduce launch per segment (host offsets)."""
    import torch
    nseg = len(h_offsets) - 1
    if out is None:
        out = torch.empty_like(x)
    if sums is None:
        sums = torch.empty(nseg, dtype=x.dtype, device=x.device)
    if ws is None:
        ws = desc_segmented_workspace(nseg, x.numel(), x.device)
    arr = (c_int64 * len(h_offsets))(*[int(v) for v in h_offsets])
    _check(lib().desc_segmented_reduce_scan_per_segment(arr, nseg, _dtype_code(x), _ptr(x), _ptr(out), _ptr(sums),
                                                        _ptr(ws), ws.numel(), _stream(stream)),
           "desc_segmented_reduce_scan_per_segment")
    return out, sums


def desc_scan_noalloc(x, base_shape, ops, seg_level, grid=None, block=None, out=None, stream=None):
    """desc_scan without a workspace: the library's static scratch is used
    (contiguous scans of at most 2^28 elements; calls must not overlap)."""
    import torch
    if out is None:
        out = torch.empty_like(x)
    _check(lib().desc_scan_noalloc(ctypes.byref(make_view(base_shape, ops)), _ref(make_exec(grid, block)), seg_level,
                                   _dtype_code(x), _ptr(x), x.numel() * 4, _ptr(out), out.numel() * 4,
                                   _stream(stream)), "desc_scan_noalloc")
    return out


def desc_stream_status(stream=None) -> int:
    return lib().desc_stream_status(_stream(stream))


# ----------------------------------------------------------------- schedules
class ProblemRef:
    """A desc_problem and the host arrays it points to (kept alive with it)."""

    def __init__(self, prob: dict):
        p = Problem()
        p.op, p.dtype, p.n, p.aux = int(prob["op"]), int(prob["dtype"]), int(prob["n"]), int(prob.get("aux", 0))
        p.k = int(prob.get("k", 0) or 0)
        self.keep = []
        lengths = prob.get("lengths")
        if lengths is not None:
            vals = lengths.tolist() if hasattr(lengths, "tolist") else list(lengths)
            arr = (c_int64 * max(len(vals), 1))(*[int(v) for v in vals])
            self.keep.append(arr)
            p.seg_lengths = ctypes.cast(arr, POINTER(c_int64))
        if prob.get("view") is not None:
            base_shape, ops = prob["view"]
            v = make_view(base_shape, ops)
            self.keep.append(v)
            p.view = ctypes.pointer(v)
            if prob.get("grid") is not None:
                e = make_exec(prob["grid"], prob["block"])
                self.keep.append(e)
                p.ex = ctypes.pointer(e)
            p.level = int(prob.get("level", GRID))
        self.p = p

    def ref(self):
        return ctypes.byref(self.p)


def make_problem(op, dtype, n, aux=0, lengths=None, k=0, view=None, grid=None, block=None, level=GRID) -> ProblemRef:
    """Matmul: n = M, aux = N, k = K.  view = (base_shape, ops) for a reduce or
    scan through that view (grid / block its resource, level its out_level /
    seg_level)."""
    return ProblemRef(dict(op=op, dtype=dtype, n=n, aux=aux, lengths=lengths, k=k, view=view, grid=grid,
                           block=block, level=level))


def _problem(prob) -> ProblemRef:
    return prob if isinstance(prob, ProblemRef) else ProblemRef(prob)


def candidate_count(op) -> int:
    c = c_int32(0)
    _check(lib().desc_candidate_count(int(op), ctypes.byref(c)), "desc_candidate_count")
    return c.value


def desc_features(problem, cand: int):
    out = (ctypes.c_float * NUM_FEATURES)()
    _check(lib().desc_features(_problem(problem).ref(), int(cand), out, NUM_FEATURES), "desc_features")
    return list(out)


def desc_force_candidate(op, cand):
    _check(lib().desc_force_candidate(int(op), int(cand)), "desc_force_candidate")


def desc_force_generic(on):
    """Evaluate this thread's reduce / scan / transpose views through the
    general affine-map kernels (the view-overhead experiment's other arm)."""
    _check(lib().desc_force_generic(1 if on else 0), "desc_force_generic")


def desc_tune_record(problem, cand):
    _check(lib().desc_tune_record(_problem(problem).ref(), int(cand)), "desc_tune_record")


def desc_tune_lookup(problem):
    c = c_int32(-1)
    _check(lib().desc_tune_lookup(_problem(problem).ref(), ctypes.byref(c)), "desc_tune_lookup")
    return c.value


def desc_tune_clear():
    _check(lib().desc_tune_clear(), "desc_tune_clear")


def desc_tune_save(path):
    _check(lib().desc_tune_save(str(path).encode()), "desc_tune_save")


def desc_tune_load(path):
    _check(lib().desc_tune_load(str(path).encode()), "desc_tune_load")


class TuneArena:
    """Device buffers the tuner measures on (the largest problem decides);
    max_mm > 0 adds room for matmul problems up to M = N = K = max_mm."""

    def __init__(self, max_n, max_seg, device="cuda", max_mm=0):
        import torch
        max_n = max(max_n, max_mm * max_mm)
        self.x = torch.zeros(max_n, dtype=torch.float32, device=device)
        self.y = torch.zeros(max_n, dtype=torch.float32, device=device)
        self.b = torch.zeros(max(max_mm * max_mm, 1), dtype=torch.float32, device=device)
        self.sums = torch.zeros(max(max_seg, 1), dtype=torch.float32, device=device)
        self.offsets = torch.zeros(max_seg + 1, dtype=torch.int64, device=device)
        nb = max(desc_segmented_workspace(max_seg, max_n, "cpu").numel(), 1 << 20)
        nb2 = c_size_t(0)
        _check(lib().desc_scan_workspace_size(ctypes.byref(make_view([max_n], [])), None, GRID, F32,
                                              ctypes.byref(nb2)), "desc_scan_workspace_size")
        nb3 = c_size_t(0)
        if max_mm:
            _check(lib().desc_matmul_workspace_size(max_mm, max_mm, max_mm, MM_BF16, ctypes.byref(nb3)),
                   "desc_matmul_workspace_size")
        self.ws = torch.empty(max(nb, nb2.value, nb3.value) + (64 << 20), dtype=torch.uint8, device=device)

    def buffers(self, prob: dict):
        import torch
        b = TuneBuffers()
        b.inp, b.out, b.sums = self.x.data_ptr(), self.y.data_ptr(), self.sums.data_ptr()
        b.ws, b.ws_bytes = self.ws.data_ptr(), self.ws.numel()
        b.in2 = self.b.data_ptr()
        if prob["op"] == OP_SEGMENTED:
            L = prob["lengths"]
            off = torch.zeros(L.numel() + 1, dtype=torch.int64)
            off[1:] = torch.cumsum(L.to(torch.int64), 0)
            self.offsets[: off.numel()].copy_(off)
        b.offsets = self.offsets.data_ptr()
        return b


def desc_tune_measure(prob: dict, arena: TuneArena, reps=5, stream=None):
    p = _problem(prob)
    nc = candidate_count(prob["op"])
    us = (ctypes.c_float * nc)()
    _check(lib().desc_tune_measure(p.ref(), ctypes.byref(arena.buffers(prob)), int(reps), _stream(stream), us),
           "desc_tune_measure")
    return list(us)


def desc_tune_measure_cands(prob: dict, arena: TuneArena, cands, reps=20, stream=None):
    """Times the listed candidates in interleaved rounds (median of reps)."""
    p = _problem(prob)
    arr = (c_int32 * len(cands))(*[int(c) for c in cands])
    us = (ctypes.c_float * len(cands))()
    _check(lib().desc_tune_measure_cands(p.ref(), ctypes.byref(arena.buffers(prob)), arr, len(cands), int(reps),
                                         _stream(stream), us), "desc_tune_measure_cands")
    return list(us)


def desc_tune_exhaustive(prob: dict, arena: TuneArena, reps=5, stream=None):
    p = _problem(prob)
    best = c_int32(-1)
    _check(lib().desc_tune_exhaustive(p.ref(), ctypes.byref(arena.buffers(prob)), int(reps), _stream(stream),
                                      ctypes.byref(best)), "desc_tune_exhaustive")
    return best.value


class CostModel:
    """The schedule cost model: FP32 parameters, Adam moments and workspace on
    the device; forward, backward, Adam and the picker run in libdesc."""

    def __init__(self, params, F=NUM_FEATURES, H=64):
        import torch
        self.F, self.H = F, H
        self.p = params.to("cuda", torch.float32).contiguous().clone()
        self.m = torch.zeros_like(self.p)
        self.v = torch.zeros_like(self.p)
        self.g = torch.zeros_like(self.p)

    def _ws(self, rows):
        import torch
        nb = c_size_t(0)
        _check(lib().desc_mlp_workspace_size(self.F, self.H, int(rows), ctypes.byref(nb)), "desc_mlp_workspace_size")
        return torch.empty(max(nb.value, 4), dtype=torch.uint8, device="cuda")

    def forward(self, X):
        import torch
        y = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
        _check(lib().desc_mlp_forward(_ptr(self.p), self.F, self.H, _ptr(X), X.shape[0], _ptr(y), None, 0,
                                      _stream(None)), "desc_mlp_forward")
        return y

    def backward(self, X, t):
        ws = self._ws(X.shape[0])
        _check(lib().desc_mlp_backward(_ptr(self.p), self.F, self.H, _ptr(X), _ptr(t), X.shape[0], _ptr(self.g),
                                       _ptr(ws), ws.numel(), _stream(None)), "desc_mlp_backward")
        return self.g

    def adam(self, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(lib().desc_mlp_adam(_ptr(self.p), _ptr(self.g), _ptr(self.m), _ptr(self.v), self.p.numel(), int(step),
                                   lr, beta1, beta2, eps, _stream(None)), "desc_mlp_adam")

    def train(self, X, t, epochs, batch, lr):
        ws = self._ws(X.shape[0])
        loss = ctypes.c_float(0)
        _check(lib().desc_mlp_train(_ptr(self.p), _ptr(self.g), _ptr(self.m), _ptr(self.v), self.F, self.H, _ptr(X),
                                    _ptr(t), X.shape[0], int(epochs), int(batch), float(lr), _ptr(ws), ws.numel(),
                                    _stream(None), ctypes.byref(loss)), "desc_mlp_train")
        return loss.value

    def pick(self, Xcand):
        import torch
        pred = torch.empty(Xcand.shape[0], dtype=torch.float32, device="cuda")
        best = torch.empty(1, dtype=torch.int32, device="cuda")
        _check(lib().desc_mlp_pick(_ptr(self.p), self.F, self.H, _ptr(Xcand), Xcand.shape[0], _ptr(pred), _ptr(best),
                                   _stream(None)), "desc_mlp_pick")
        return int(best.item()), pred

    def install(self):
        """Use this model for desc_tune_predict (kept by reference)."""
        _check(lib().desc_tune_set_model(_ptr(self.p), self.F, self.H), "desc_tune_set_model")

    def predict_problem(self, prob, stream=None):
        best = c_int32(-1)
        _check(lib().desc_tune_predict(_problem(prob).ref(), _stream(stream), ctypes.byref(best)),
               "desc_tune_predict")
        return best.value


def feature_rows(prob):
    p = _problem(prob)
    return [desc_features(p, c) for c in range(candidate_count(p.p.op))]
