// Entry points of libdesc: validate, lower the views, check accesses, pick
// a schedule from the lowered maps, and launch.  Nothing is launched before
// every check has passed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "desc_internal.h"

namespace desc {

int32_t check_device_ptr(const void *p, size_t align) {
  if (!p) return DESC_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(p) % align) return DESC_ERR_ALIGNMENT;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return DESC_ERR_HOST_POINTER;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return DESC_OK;
  return DESC_ERR_HOST_POINTER;
}

}  // namespace desc

using namespace desc;

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return na && nb && x < y + nb && y < x + na;
}

// Write map of one op: with selects, no element may be written by two
// logical threads (desc_check_disjoint).  The kernels write in parallel, so
// an element reached twice by the same logical thread cannot keep its
// write order either: such maps are not supported.
int32_t check_writes(const desc_lowered &w, const desc_exec *ex) {
  if (ex) {
    desc_access a;
    a.map = w;
    a.buffer = 0;
    a.is_write = 1;
    int64_t first = 0;
    const int32_t r = desc_check_disjoint(&a, 1, ex, &first);
    if (r != DESC_OK) return r;
  }
  return injective_quick(w) ? DESC_OK : DESC_ERR_UNSUPPORTED;
}

}  // namespace

// Per-thread switch: evaluate every view through the general affine kernels.
namespace {
thread_local bool t_generic = false;
}
extern "C" int32_t desc_force_generic(int32_t on) {
  t_generic = on != 0;
  return DESC_OK;
}

// ---------------------------------------------------------------- reduce
extern "C" int32_t desc_reduce_workspace_size(const desc_view *v, const desc_exec *ex,
                                              int32_t out_level, int32_t dtype, size_t *bytes) {
  if (!bytes || !dtype_size(dtype)) return DESC_ERR_INVALID_ARG;
  if (out_level < DESC_LEVEL_GRID || out_level > DESC_LEVEL_THREAD) return DESC_ERR_INVALID_ARG;
  desc_lowered L;
  int32_t r = desc_lower_view(v, ex, &L);
  if (r != DESC_OK) return r;
  const Plan p = split_plan(L, out_level);
  int64_t start0, seg;
  *bytes = (!t_generic && rest_contiguous(p, true, &start0, &seg)) ? reduce_segments_ws(dtype, p.n_rest, p.n_keep)
                                                                   : reduce_affine_ws(p.n_rest, p.n_keep);
  return DESC_OK;
}

extern "C" int32_t desc_reduce(const desc_view *v, const desc_exec *ex, int32_t out_level,
                               int32_t dtype, const void *in, size_t in_bytes, void *out,
                               size_t out_bytes, int32_t flags, void *ws, size_t ws_bytes,
                               desc_stream_t s) {
  if (!dtype_size(dtype)) return DESC_ERR_INVALID_ARG;
  if (out_level < DESC_LEVEL_GRID || out_level > DESC_LEVEL_THREAD) return DESC_ERR_INVALID_ARG;
  if (flags & ~kOperatorFlags) return DESC_ERR_INVALID_ARG;
  if (check_operator(flags, dtype, false) != DESC_OK) return DESC_ERR_INVALID_ARG;
  desc_lowered L;
  int32_t r = desc_lower_view(v, ex, &L);
  if (r != DESC_OK) return r;
  if ((flags & kArgFlags) && L.base_elems >= (int64_t(1) << 31)) return DESC_ERR_UNSUPPORTED;   // int32 indices
  const Plan p = split_plan(L, out_level);
  if (in_bytes != size_t(L.base_elems) * 4 || out_bytes != size_t(p.n_keep) * 4)
    return DESC_ERR_SIZE_MISMATCH;
  if (p.n_keep == 0) return DESC_OK;
  if ((r = check_device_ptr(out, 4)) != DESC_OK) return r;
  if (L.base_elems > 0 && (r = check_device_ptr(in, 4)) != DESC_OK) return r;
  if (ranges_overlap(in, in_bytes, out, out_bytes)) return DESC_ERR_OVERLAP;
  if (p.n_rest == 0) return fill_identity(out, p.n_keep, dtype, flags, s);
  int64_t start0, seg;
  if (!t_generic && rest_contiguous(p, true, &start0, &seg))
    return launch_reduce_segments(dtype, in, start0, seg, p.n_rest, p.n_keep, out, flags, ws,
                                  ws_bytes, s,
                                  schedule_for(DESC_OP_REDUCE, dtype, p.n_rest * p.n_keep,
                                               p.n_keep > 1 ? p.n_keep : 0));
  return launch_reduce_affine(dtype, in, p, out, flags, ws, ws_bytes, s);
}

// ---------------------------------------------------------------- split launch
extern "C" int32_t desc_split_reduce_transpose(const desc_view *rv, const desc_exec *rex, int32_t out_level,
                                               int32_t dtype, const void *rin, size_t rin_bytes, void *rout,
                                               size_t rout_bytes, void *ws, size_t ws_bytes, const float *tin,
                                               float *tout, int64_t R, int64_t C, desc_stream_t s) {
  if (!dtype_size(dtype) || R < 0 || C < 0) return DESC_ERR_INVALID_ARG;
  if (out_level < DESC_LEVEL_GRID || out_level > DESC_LEVEL_THREAD) return DESC_ERR_INVALID_ARG;
  desc_lowered L;
  int32_t r = desc_lower_view(rv, rex, &L);
  if (r != DESC_OK) return r;
  const Plan p = split_plan(L, out_level);
  if (rin_bytes != size_t(L.base_elems) * 4 || rout_bytes != size_t(p.n_keep) * 4) return DESC_ERR_SIZE_MISMATCH;
  int64_t start0, seg;
  if (p.n_keep == 0 || p.n_rest == 0 || !rest_contiguous(p, true, &start0, &seg)) return DESC_ERR_UNSUPPORTED;
  const size_t tb = size_t(R) * size_t(C) * 4;
  if ((r = check_device_ptr(rout, 4)) != DESC_OK || (r = check_device_ptr(rin, 4)) != DESC_OK) return r;
  if (tb && ((r = check_device_ptr(tin, 4)) != DESC_OK || (r = check_device_ptr(tout, 4)) != DESC_OK)) return r;
  const void *bufs[4] = {rin, rout, tin, tout};
  const size_t sizes[4] = {rin_bytes, rout_bytes, tb, tb};
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j)
      if (ranges_overlap(bufs[i], sizes[i], bufs[j], sizes[j])) return DESC_ERR_OVERLAP;
  return launch_split_reduce_transpose(dtype, rin, start0, seg, p.n_rest, p.n_keep, rout, ws, ws_bytes, tin, tout,
                                       R, C, s);
}

// ---------------------------------------------------------------- scan
namespace {

struct ScanPlan {
  bool contig;       // fast path: one contiguous run [start, start + total)
  int64_t start, total, period;
};

ScanPlan plan_scan(const desc_lowered &L, int32_t seg_level) {
  const Plan p = split_plan(L, seg_level);
  ScanPlan sp{false, 0, p.n_keep * p.n_rest, p.n_rest};
  int64_t start0, seg;
  if (!t_generic && rest_contiguous(p, false, &start0, &seg) && (p.n_keep <= 1 || seg == p.n_rest)) {
    sp.contig = true;
    sp.start = start0;
  }
  return sp;
}

}  // namespace

extern "C" int32_t desc_scan_workspace_size(const desc_view *v, const desc_exec *ex,
                                            int32_t seg_level, int32_t dtype, size_t *bytes) {
  if (!bytes || !dtype_size(dtype)) return DESC_ERR_INVALID_ARG;
  if (seg_level < DESC_LEVEL_GRID || seg_level > DESC_LEVEL_THREAD) return DESC_ERR_INVALID_ARG;
  desc_lowered L;
  int32_t r = desc_lower_view(v, ex, &L);
  if (r != DESC_OK) return r;
  const ScanPlan sp = plan_scan(L, seg_level);
  *bytes = scan_contig_ws(dtype, sp.total);            // both scans: one tile state per 4096 points
  return DESC_OK;
}

extern "C" int32_t desc_scan(const desc_view *v, const desc_exec *ex, int32_t seg_level,
                             int32_t dtype, const void *in, size_t in_bytes, void *out,
                             size_t out_bytes, int32_t flags, void *ws, size_t ws_bytes,
                             desc_stream_t s) {
  if (!dtype_size(dtype)) return DESC_ERR_INVALID_ARG;
  if (seg_level < DESC_LEVEL_GRID || seg_level > DESC_LEVEL_THREAD) return DESC_ERR_INVALID_ARG;
  if (flags & ~(DESC_DEBUG_STALL_TILE | DESC_EXCLUSIVE | kOperatorFlags)) return DESC_ERR_INVALID_ARG;
  if (check_operator(flags, dtype, true) != DESC_OK) return DESC_ERR_INVALID_ARG;
  desc_lowered L;
  int32_t r = desc_lower_view(v, ex, &L);
  if (r != DESC_OK) return r;
  if (in_bytes != size_t(L.base_elems) * 4 || out_bytes != in_bytes) return DESC_ERR_SIZE_MISMATCH;
  if ((flags & kArgFlags) && L.base_elems >= (int64_t(1) << 30) - 1) return DESC_ERR_UNSUPPORTED;
  const ScanPlan sp = plan_scan(L, seg_level);
  if (sp.total == 0) return DESC_OK;
  if ((r = check_device_ptr(in, 4)) != DESC_OK) return r;
  if ((r = check_device_ptr(out, 4)) != DESC_OK) return r;
  if (in != out && ranges_overlap(in, in_bytes, out, out_bytes)) return DESC_ERR_OVERLAP;
  if ((r = check_writes(L, ex)) != DESC_OK) return r;
  if (sp.contig) {
    const char *ib = static_cast<const char *>(in);
    char *ob = static_cast<char *>(out);
    if (flags & kArgFlags)                             // arg operators: element indices from sp.start
      return launch_scan_arg(dtype, ib + sp.start * 4, ob + sp.start * 4, sp.total, sp.period, nullptr, 0, nullptr,
                             sp.start, flags, ws, ws_bytes, s);
    return launch_scan_contig(dtype, ib + sp.start * 4, ob + sp.start * 4, sp.total, sp.period, flags, ws,
                              ws_bytes, s, schedule_for(DESC_OP_SCAN, dtype, sp.total, 0));
  }
  // one pass through the lowered map: loads gather, stores scatter
  if (!(flags & kMapScanOps))
    return launch_scan_mapped(dtype, in, out, L.offset, L.extent, L.stride, L.ndims, sp.period, flags, ws, ws_bytes,
                              s);
  return launch_scan_arg_mapped(dtype, in, out, L.offset, L.extent, L.stride, L.ndims, sp.period, flags, ws, ws_bytes,
                                s);
}

// ---------------------------------------------------------------- scan, no allocation
extern "C" int32_t desc_scan_noalloc(const desc_view *v, const desc_exec *ex, int32_t seg_level,
                                     int32_t dtype, const void *in, size_t in_bytes, void *out,
                                     size_t out_bytes, desc_stream_t s) {
  if (!dtype_size(dtype)) return DESC_ERR_INVALID_ARG;
  if (seg_level < DESC_LEVEL_GRID || seg_level > DESC_LEVEL_THREAD) return DESC_ERR_INVALID_ARG;
  desc_lowered L;
  int32_t r = desc_lower_view(v, ex, &L);
  if (r != DESC_OK) return r;
  if (in_bytes != size_t(L.base_elems) * 4 || out_bytes != in_bytes) return DESC_ERR_SIZE_MISMATCH;
  const ScanPlan sp = plan_scan(L, seg_level);
  if (sp.total == 0) return DESC_OK;
  if (!sp.contig) return DESC_ERR_UNSUPPORTED;
  if (sp.total > DESC_SCAN_NOALLOC_MAX_ELEMS) return DESC_ERR_WORKSPACE;
  if ((r = check_device_ptr(in, 4)) != DESC_OK) return r;
  if ((r = check_device_ptr(out, 4)) != DESC_OK) return r;
  if (in != out && ranges_overlap(in, in_bytes, out, out_bytes)) return DESC_ERR_OVERLAP;
  if ((r = check_writes(L, ex)) != DESC_OK) return r;
  const char *ib = static_cast<const char *>(in);
  char *ob = static_cast<char *>(out);
  return launch_scan_contig_noalloc(dtype, ib + sp.start * 4, ob + sp.start * 4, sp.total,
                                    sp.period, s);
}

// ---------------------------------------------------------------- transpose
extern "C" int32_t desc_transpose(const desc_view *in_v, const desc_view *out_v,
                                  const desc_exec *ex, int32_t dtype, const void *in,
                                  size_t in_bytes, void *out, size_t out_bytes, desc_stream_t s) {
  if (!dtype_size(dtype)) return DESC_ERR_INVALID_ARG;
  desc_lowered Li, Lo;
  int32_t r;
  if ((r = desc_lower_view(in_v, ex, &Li)) != DESC_OK) return r;
  if ((r = desc_lower_view(out_v, ex, &Lo)) != DESC_OK) return r;
  if (!ex && (Li.nsel || Lo.nsel)) return DESC_ERR_INVALID_ARG;
  if (Li.ndims != Lo.ndims || Li.nsel != Lo.nsel) return DESC_ERR_SHAPE;
  for (int i = 0; i < Li.ndims; ++i)
    if (Li.extent[i] != Lo.extent[i] || Li.level[i] != Lo.level[i] || Li.dim[i] != Lo.dim[i])
      return DESC_ERR_SHAPE;
  if (in_bytes != size_t(Li.base_elems) * 4 || out_bytes != size_t(Lo.base_elems) * 4)
    return DESC_ERR_SIZE_MISMATCH;
  int64_t total = 1;
  for (int i = 0; i < Li.ndims; ++i) total *= Li.extent[i];
  if (total == 0) return DESC_OK;
  if ((r = check_device_ptr(in, 4)) != DESC_OK) return r;
  if ((r = check_device_ptr(out, 4)) != DESC_OK) return r;
  // In place, the parallel copy would read elements other threads have
  // already overwritten unless both views reach the same element per point.
  if (in == out) {
    if (!same_map_quick(Li, Lo)) return DESC_ERR_OVERLAP;
  } else if (ranges_overlap(in, in_bytes, out, out_bytes)) {
    return DESC_ERR_OVERLAP;
  }
  if ((r = check_writes(Lo, ex)) != DESC_OK) return r;

  // canonical dims: (extent, in stride, out stride), output-major order
  struct D { int64_t e, si, so; };
  std::vector<D> d;
  for (int i = 0; i < Li.ndims; ++i)
    if (Li.extent[i] > 1) d.push_back({Li.extent[i], Li.stride[i], Lo.stride[i]});
  bool pos = !t_generic;
  for (auto &x : d) pos = pos && x.so > 0;
  if (pos) {
    std::sort(d.begin(), d.end(), [](const D &a, const D &b) { return a.so > b.so; });
    std::vector<D> m;
    for (auto &x : d) {
      if (!m.empty() && m.back().si == x.si * x.e && m.back().so == x.so * x.e) {
        m.back().e *= x.e;
        m.back().si = x.si;
        m.back().so = x.so;
      } else {
        m.push_back(x);
      }
    }
    // [batch] x (C: out-major, in-stride 1) x (R: out-stride 1, in-stride ld_in)
    const size_t k = m.size();
    if ((k == 2 || k == 3) && m[k - 1].so == 1 && m[k - 2].si == 1) {
      const int64_t R = m[k - 1].e, C = m[k - 2].e, ld_in = m[k - 1].si, ld_out = m[k - 2].so;
      const int64_t batch = k == 3 ? m[0].e : 1, bs_in = k == 3 ? m[0].si : 0,
                    bs_out = k == 3 ? m[0].so : 0;
      if (ld_in >= C && ld_out >= R)
        return launch_transpose(static_cast<const float *>(in) + Li.offset,
                                static_cast<float *>(out) + Lo.offset, R, C, ld_in, ld_out, batch,
                                bs_in, bs_out, s,
                                schedule_for(DESC_OP_TRANSPOSE, dtype, R * C, R));
    }
  }
  return launch_copy_affine(in, Li.offset, Li.stride, out, Lo.offset, Lo.stride, Li.extent,
                            Li.ndims, s);
}

// ---------------------------------------------------------------- matmul
namespace {

// Lowered 2-D operand map: extents (r, c), strides, offset.
int32_t operand_map(const desc_view *v, int64_t R, int64_t Cc, int64_t *off, int64_t *sr, int64_t *sc,
                    int64_t *elems) {
  if (!v) {
    *off = 0; *sr = Cc; *sc = 1; *elems = R * Cc;
    return DESC_OK;
  }
  desc_lowered L;
  const int32_t r = desc_lower_view(v, nullptr, &L);
  if (r != DESC_OK) return r;
  if (L.nsel != 0 || L.ndims != 2 || L.extent[0] != R || L.extent[1] != Cc) return DESC_ERR_SHAPE;
  *off = L.offset; *sr = L.stride[0]; *sc = L.stride[1]; *elems = L.base_elems;
  return DESC_OK;
}

int mm_planes(int32_t precision) {
  switch (precision) {
    case DESC_MM_BF16: return 1;
    case DESC_MM_SPLIT2: return 2;
    case DESC_MM_SPLIT3: return 3;
    default: return 0;
  }
}

}  // namespace

extern "C" int32_t desc_matmul_workspace_size(int64_t M, int64_t N, int64_t K, int32_t precision,
                                              size_t *bytes) {
  if (!bytes || M < 0 || N < 0 || K < 0) return DESC_ERR_INVALID_ARG;
  if (precision == DESC_MM_FP32_SIMT) { *bytes = 0; return DESC_OK; }
  const int planes = mm_planes(precision);
  if (!planes) return DESC_ERR_INVALID_ARG;
  *bytes = mm_tc_ws(M, N, K, planes);
  return DESC_OK;
}

extern "C" int32_t desc_matmul_plan(int64_t M, int64_t N, int64_t K, int32_t precision, int32_t candidate,
                                    int32_t max_pairs, desc_mm_plan *plan) {
  const int planes = mm_planes(precision);
  if (!plan || !planes || M <= 0 || N <= 0 || K <= 0 || candidate < -1 || candidate >= mm_candidates() ||
      max_pairs < 0)
    return DESC_ERR_INVALID_ARG;
  if (max_pairs == 0 && (max_pairs = mm_max_pairs()) <= 0) return DESC_ERR_CUDA;
  const int nprod = planes == 3 ? 6 : (planes == 2 ? 3 : 1);
  MmPlan pl;
  const int32_t r = mm_plan(M, N, K, nprod, candidate >= 0 ? candidate : schedule_for(DESC_OP_MATMUL, DESC_F32, M, N),
                            max_pairs, &pl);
  if (r != DESC_OK) return r;
  plan->candidate = pl.cand;
  plan->pairs = pl.pairs;
  plan->tile_n = 256 * pl.width;
  plan->padded = pl.padded;
  plan->rows = pl.Mp;
  plan->tiles = pl.tiles;
  plan->whole_tiles = pl.whole;
  plan->pieces = pl.pieces;
  plan->max_pairs = max_pairs;
  return DESC_OK;
}

extern "C" int32_t desc_matmul(const desc_view *a_v, const desc_view *b_v, int64_t M, int64_t N, int64_t K,
                               const float *A, size_t a_bytes, const float *B, size_t b_bytes, float *C,
                               size_t c_bytes, int32_t precision, void *ws, size_t ws_bytes, desc_stream_t s) {
  if (M < 0 || N < 0 || K < 0) return DESC_ERR_INVALID_ARG;
  if (precision != DESC_MM_FP32_SIMT && !mm_planes(precision)) return DESC_ERR_INVALID_ARG;
  int64_t ao, asr, asc, ae, bo, bsr, bsc, be;
  int32_t r;
  if ((r = operand_map(a_v, M, K, &ao, &asr, &asc, &ae)) != DESC_OK) return r;
  if ((r = operand_map(b_v, K, N, &bo, &bsr, &bsc, &be)) != DESC_OK) return r;
  if (a_bytes != size_t(ae) * 4 || b_bytes != size_t(be) * 4 || c_bytes != size_t(M) * N * 4)
    return DESC_ERR_SIZE_MISMATCH;
  if (M == 0 || N == 0) return DESC_OK;
  if ((r = check_device_ptr(C, 4)) != DESC_OK) return r;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  if (K == 0) return cudaMemsetAsync(C, 0, c_bytes, st) == cudaSuccess ? DESC_OK : DESC_ERR_CUDA;
  if ((r = check_device_ptr(A, 4)) != DESC_OK) return r;
  if ((r = check_device_ptr(B, 4)) != DESC_OK) return r;
  if (ranges_overlap(A, a_bytes, C, c_bytes) || ranges_overlap(B, b_bytes, C, c_bytes)) return DESC_ERR_OVERLAP;
  if (precision == DESC_MM_FP32_SIMT) {
    if (asc != 1 || bsc != 1 || asr < 0 || bsr < 0) return DESC_ERR_UNSUPPORTED;
    return launch_sgemm(A + ao, B + bo, C, M, N, K, asr, bsr, N, s);
  }
  // products in increasing order of magnitude (the largest, A_0 B_0, last)
  static const int pa3[6] = {2, 1, 0, 1, 0, 0}, pb3[6] = {0, 1, 2, 0, 1, 0};
  static const int pa2[3] = {1, 0, 0}, pb2[3] = {0, 1, 0};
  static const int pa1[1] = {0}, pb1[1] = {0};
  const int planes = mm_planes(precision);
  const int nprod = planes == 3 ? 6 : (planes == 2 ? 3 : 1);
  const int *pa = planes == 3 ? pa3 : (planes == 2 ? pa2 : pa1);
  const int *pb = planes == 3 ? pb3 : (planes == 2 ? pb2 : pb1);
  return launch_mm_tc(A, ao, asr, asc, B, bo, bsr, bsc, C, M, N, K, planes, nprod, pa, pb, ws, ws_bytes, s);
}

// ---------------------------------------------------------------- segmented
namespace {

int32_t check_offsets_host(const int64_t *h, int64_t nseg, int64_t total) {
  if (h[0] != 0 || h[nseg] != total) return DESC_ERR_SHAPE;
  for (int64_t i = 0; i < nseg; ++i)
    if (h[i + 1] < h[i]) return DESC_ERR_SHAPE;
  return DESC_OK;
}

int32_t check_offsets_device(const int64_t *d, int64_t nseg, int64_t total) {
  std::vector<int64_t> h(size_t(nseg) + 1);
  if (cudaMemcpy(h.data(), d, h.size() * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return DESC_ERR_CUDA;
  return check_offsets_host(h.data(), nseg, total);
}

int32_t segmented_checks(const int64_t *d_offsets, int64_t nseg, int64_t total, int32_t dtype, const void *in,
                         void *scan_out, void *sums_out) {
  if (nseg < 0 || total < 0 || !dtype_size(dtype)) return DESC_ERR_INVALID_ARG;
  int32_t r;
  if ((r = check_device_ptr(d_offsets, 8)) != DESC_OK) return r;
  if (nseg > 0 && (r = check_device_ptr(sums_out, 4)) != DESC_OK) return r;
  if (total > 0) {
    if ((r = check_device_ptr(in, 4)) != DESC_OK) return r;
    if ((r = check_device_ptr(scan_out, 4)) != DESC_OK) return r;
  }
  const size_t tb = size_t(total) * 4, sb = size_t(nseg) * 4;
  if (in != scan_out && ranges_overlap(in, tb, scan_out, tb)) return DESC_ERR_OVERLAP;
  if (ranges_overlap(sums_out, sb, scan_out, tb) || ranges_overlap(sums_out, sb, in, tb) ||
      ranges_overlap(d_offsets, size_t(nseg + 1) * 8, scan_out, tb) ||
      ranges_overlap(d_offsets, size_t(nseg + 1) * 8, sums_out, sb))
    return DESC_ERR_OVERLAP;
  return DESC_OK;
}

}  // namespace

struct desc_graph_st {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

extern "C" int32_t desc_segmented_workspace_size(int64_t nseg, int64_t total, size_t *bytes) {
  if (!bytes || nseg < 0 || total < 0) return DESC_ERR_INVALID_ARG;
  *bytes = scan_csr_ws(total);
  return DESC_OK;
}

extern "C" int32_t desc_segmented_reduce_scan(const int64_t *d_offsets, int64_t nseg, int64_t total,
                                              int32_t dtype, const void *in, void *scan_out, void *sums_out,
                                              int32_t flags, void *ws, size_t ws_bytes, desc_stream_t s) {
  if (flags & ~(DESC_CHECK_OFFSETS | DESC_DEBUG_STALL_TILE | DESC_EXCLUSIVE | kOperatorFlags))
    return DESC_ERR_INVALID_ARG;
  if (check_operator(flags, dtype, true) != DESC_OK) return DESC_ERR_INVALID_ARG;
  if ((flags & kArgFlags) && total >= (int64_t(1) << 30) - 1) return DESC_ERR_UNSUPPORTED;
  int32_t r = segmented_checks(d_offsets, nseg, total, dtype, in, scan_out, sums_out);
  if (r != DESC_OK) return r;
  if (nseg == 0) return total == 0 ? DESC_OK : DESC_ERR_SHAPE;
  if ((flags & DESC_CHECK_OFFSETS) && (r = check_offsets_device(d_offsets, nseg, total)) != DESC_OK) return r;
  if (total == 0) return fill_identity(sums_out, nseg, dtype, flags, s);   // every segment is empty
  const int32_t kf = flags & (DESC_DEBUG_STALL_TILE | DESC_EXCLUSIVE | kOperatorFlags);
  if (flags & kArgFlags) {                             // empty segments keep the identity written first
    if ((r = fill_identity(sums_out, nseg, dtype, flags, s)) != DESC_OK) return r;
    return launch_scan_arg(dtype, in, scan_out, total, 0, d_offsets, nseg, sums_out, 0, kf, ws, ws_bytes, s);
  }
  return launch_scan_csr(dtype, in, scan_out, total, d_offsets, nseg, sums_out, kf, ws, ws_bytes, s,
                         schedule_for(DESC_OP_SEGMENTED, dtype, total, nseg));
}

extern "C" int32_t desc_segmented_graph_create(const int64_t *d_offsets, int64_t nseg, int64_t total,
                                               int32_t dtype, const void *in, void *scan_out, void *sums_out,
                                               void *ws, size_t ws_bytes, desc_graph_t *graph) {
  if (!graph) return DESC_ERR_INVALID_ARG;
  int32_t r = segmented_checks(d_offsets, nseg, total, dtype, in, scan_out, sums_out);
  if (r != DESC_OK) return r;
  if (nseg == 0) return DESC_ERR_SHAPE;
  if ((r = check_offsets_device(d_offsets, nseg, total)) != DESC_OK) return r;
  if (total > 0 && (!ws || ws_bytes < scan_csr_ws(total))) return DESC_ERR_WORKSPACE;
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return DESC_ERR_CUDA;
  desc_graph_st *g = new desc_graph_st{nullptr, nullptr};
  r = DESC_OK;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) r = DESC_ERR_CUDA;
  if (r == DESC_OK) {
    const int32_t lr = desc_segmented_reduce_scan(d_offsets, nseg, total, dtype, in, scan_out, sums_out, 0, ws,
                                                  ws_bytes, reinterpret_cast<desc_stream_t>(cs));
    const cudaError_t e = cudaStreamEndCapture(cs, &g->graph);
    if (lr != DESC_OK) r = lr;
    else if (e != cudaSuccess) r = DESC_ERR_CUDA;
  }
  if (r == DESC_OK && cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) r = DESC_ERR_CUDA;
  cudaStreamDestroy(cs);
  if (r != DESC_OK) {
    (void)cudaGetLastError();
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return r;
  }
  *graph = g;
  return DESC_OK;
}

extern "C" int32_t desc_graph_launch(desc_graph_t g, desc_stream_t s) {
  if (!g || !g->exec) return DESC_ERR_INVALID_ARG;
  return cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(s)) == cudaSuccess ? DESC_OK : DESC_ERR_CUDA;
}

extern "C" int32_t desc_graph_destroy(desc_graph_t g) {
  if (!g) return DESC_ERR_INVALID_ARG;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return DESC_OK;
}

extern "C" int32_t desc_segmented_reduce_scan_per_segment(const int64_t *h_offsets, int64_t nseg, int32_t dtype,
                                                          const void *in, void *scan_out, void *sums_out,
                                                          void *ws, size_t ws_bytes, desc_stream_t s) {
  if (!h_offsets || nseg < 0 || !dtype_size(dtype)) return DESC_ERR_INVALID_ARG;
  if (nseg == 0) return DESC_OK;
  const int64_t total = h_offsets[nseg];
  int32_t r;
  if ((r = check_offsets_host(h_offsets, nseg, total)) != DESC_OK) return r;
  if ((r = check_device_ptr(sums_out, 4)) != DESC_OK) return r;
  const char *ib = static_cast<const char *>(in);
  char *ob = static_cast<char *>(scan_out);
  char *sb = static_cast<char *>(sums_out);
  for (int64_t i = 0; i < nseg; ++i) {
    const int64_t a = h_offsets[i], len = h_offsets[i + 1] - a;
    if (len == 0) {
      if (cudaMemsetAsync(sb + i * 4, 0, 4, reinterpret_cast<cudaStream_t>(s)) != cudaSuccess) return DESC_ERR_CUDA;
      continue;
    }
    desc_view v;
    std::memset(&v, 0, sizeof(v));
    v.rank = 1;
    v.shape[0] = len;
    if ((r = desc_scan(&v, nullptr, DESC_LEVEL_GRID, dtype, ib + a * 4, size_t(len) * 4, ob + a * 4,
                       size_t(len) * 4, 0, ws, ws_bytes, s)) != DESC_OK)
      return r;
    if ((r = desc_reduce(&v, nullptr, DESC_LEVEL_GRID, dtype, ib + a * 4, size_t(len) * 4, sb + i * 4, 4, 0, ws,
                         ws_bytes, s)) != DESC_OK)
      return r;
  }
  return DESC_OK;
}

// ---------------------------------------------------------------- status
extern "C" int32_t desc_stream_status(desc_stream_t s) {
  if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(s)) != cudaSuccess) return DESC_ERR_CUDA;
  const int32_t a = scan_status_take();
  const int32_t b = mm_status_take();
  return a != DESC_OK ? a : b;
}
