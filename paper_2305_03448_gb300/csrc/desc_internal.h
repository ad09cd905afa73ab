// Internal declarations shared by the translation units of libdesc.
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/desc.h"
#include "candidates.h"

namespace desc {

// Element size of a dtype (0 when unknown).
inline size_t dtype_size(int32_t t) { return (t == DESC_I32 || t == DESC_F32) ? 4 : 0; }

// The operator flags of reduce and scan calls (at most one may be set; none
// is the sum).
constexpr int32_t kOperatorFlags = DESC_KAHAN | DESC_MAX | DESC_MIN | DESC_PROD | DESC_AND | DESC_OR | DESC_XOR |
                                   DESC_ARGMAX | DESC_ARGMIN;
constexpr int32_t kArgFlags = DESC_ARGMAX | DESC_ARGMIN;
// DESC_OK when `flags` names at most one operator and that operator applies
// to `dtype` (bitwise operators: int32 only; the compensated sum: reduces
// only, and exact anyway for int32), else DESC_ERR_INVALID_ARG.
inline int32_t check_operator(int32_t flags, int32_t dtype, bool scan) {
  const int32_t op = flags & kOperatorFlags;
  if (op & (op - 1)) return DESC_ERR_INVALID_ARG;
  if ((op & (DESC_AND | DESC_OR | DESC_XOR)) && dtype != DESC_I32) return DESC_ERR_INVALID_ARG;
  if ((op & DESC_KAHAN) && scan) return DESC_ERR_INVALID_ARG;
  return DESC_OK;
}

// A view lowered and split into the dims an op keeps (selected dims at
// levels <= a cut level, a prefix of the selected dims) and the dims it runs
// over.  Each dim: extent and stride in elements.
struct Dim {
  int64_t extent;
  int64_t stride;
};

struct Plan {
  int32_t nkeep;           // number of kept dims (prefix of the lowered dims)
  int32_t nrest;           // number of remaining dims
  Dim keep[DESC_MAX_DIMS];  // in row-major output order
  Dim rest[DESC_MAX_DIMS];  // in logical order (outermost first)
  int64_t offset;
  int64_t n_keep;          // product of kept extents (outputs or segments)
  int64_t n_rest;          // product of remaining extents
};

// Split lowered view `L` at selection level `cut`: kept dims are the selected
// dims whose level <= cut.
Plan split_plan(const desc_lowered &L, int32_t cut);

// True when the remaining dims of `p` cover one contiguous run of n_rest
// elements (in logical order, or in any order when `any_order`), and the
// runs of successive outputs start at *start0 + o * *seg_stride.
bool rest_contiguous(const Plan &p, bool any_order, int64_t *start0, int64_t *seg_stride);

// Structural injectivity of an affine map over its whole domain: sorted
// |strides| with each stride larger than the span of the smaller ones.
bool affine_injective(const int64_t *extent, const int64_t *stride, int n);

bool injective_quick(const desc_lowered &w);
bool same_map_quick(const desc_lowered &a, const desc_lowered &b);

// Pointer checks: device (or managed) memory and element alignment.
int32_t check_device_ptr(const void *p, size_t align);

// Device status words of the translation units that hold bounded waits
// (scan_status_take reads the six scan units' words).
int32_t scan_status_take();          // k_scan.cu
int32_t scan_status_take_ops();      // k_scan_ops.cu
int32_t scan_status_take_mapped();   // k_scan_mapped.cu
int32_t scan_status_take_mapped2();  // k_scan_mapped2.cu
int32_t scan_status_take_argmap();   // k_scan_arg_mapped.cu
int32_t scan_status_take_map();      // k_scan_map.cu
int32_t mm_status_take();            // k_mm_tc.cu

// ----- launchers (k_*.cu) -------------------------------------------------
// Reduce: contiguous segments [start + o*seg_stride, +len), o < nout.
// `cand`: schedule candidate (-1: the default).
int32_t launch_reduce_segments(int32_t dtype, const void *in, int64_t start, int64_t seg_stride,
                               int64_t len, int64_t nout, void *out, int32_t flags, void *ws,
                               size_t ws_bytes, desc_stream_t s, int cand);
int reduce_candidates();
size_t reduce_segments_ws(int32_t dtype, int64_t len, int64_t nout);
// Reduce: general affine plan (chunk partials in ws when runs are long).
size_t reduce_affine_ws(int64_t n_rest, int64_t nout);
// One grid: the chunked reduce of runs (sum, default schedule) on its first
// blocks, the 64 x 64 tiled transpose of an R x C FP32 matrix on the rest.
int32_t launch_split_reduce_transpose(int32_t dtype, const void *in, int64_t start, int64_t seg_stride,
                                      int64_t len, int64_t nout, void *out, void *ws, size_t ws_bytes,
                                      const float *tin, float *tout, int64_t R, int64_t C, desc_stream_t s);
// out[0 .. count) = the identity of the operator flags select (DESC_MAX,
// DESC_MIN, else the sum) in dtype.
int32_t fill_identity(void *out, int64_t count, int32_t dtype, int32_t flags, desc_stream_t s);
int32_t launch_reduce_affine(int32_t dtype, const void *in, const Plan &p, void *out,
                             int32_t flags, void *ws, size_t ws_bytes, desc_stream_t s);

// Scan of a contiguous array of n elements split into segments of length
// `period` (period == n: one segment).  in may equal out.
int32_t launch_scan_contig(int32_t dtype, const void *in, void *out, int64_t n, int64_t period,
                           int32_t flags, void *ws, size_t ws_bytes, desc_stream_t s, int cand);
int scan_candidates();
size_t scan_contig_ws(int32_t dtype, int64_t n);
// Bytes per look-back tile state: one state per 128-byte L2 line, so that the
// polls of hundreds of look-back warps spread over many L2 slices instead of
// queueing on the few lines next to the newest published prefix.
constexpr size_t kScanTileStateBytes = 128;
// The no-alloc scan always runs the 16384-element tile.
constexpr int64_t kScanNoallocTile = 16384;
// The same scan with the library's static scratch array (noalloc.cu).
int32_t launch_scan_contig_noalloc(int32_t dtype, const void *in, void *out, int64_t n,
                                   int64_t period, desc_stream_t s);
// The product and bitwise scans (k_scan_ops.cu): as launch_scan_contig /
// launch_scan_csr, default tile.
int32_t launch_scan_contig_ops(int32_t dtype, const void *in, void *out, int64_t n, int64_t period, int32_t flags,
                               void *ws, size_t ws_bytes, desc_stream_t s);
int32_t launch_scan_csr_ops(int32_t dtype, const void *in, void *out, int64_t n, const int64_t *offsets,
                            int64_t nseg, void *sums, int32_t flags, void *ws, size_t ws_bytes, desc_stream_t s);
// The arg-maximum / arg-minimum scan over one contiguous run of n points
// (segments of `period` points, or CSR offsets / nseg / sums as
// launch_scan_csr, the caller filling sums with -1 first); point g is element
// idx_base + g, whose index is written (int32).  Workspace: scan_contig_ws.
int32_t launch_scan_arg(int32_t dtype, const void *in, void *out, int64_t n, int64_t period, const int64_t *offsets,
                        int64_t nseg, void *sums, int64_t idx_base, int32_t flags, void *ws, size_t ws_bytes,
                        desc_stream_t s);
// One group of `threads` threads (32 or 256) per CSR segment (k_scan_map.cu):
// sums, maxima, minima, inclusive or exclusive; no workspace.
int32_t launch_seg_group(int32_t dtype, const void *in, void *out, const int64_t *offsets, int64_t nseg, void *sums,
                         int32_t flags, int threads, desc_stream_t s);
// Scan segmented by CSR offsets (nseg + 1 entries, device); sums (nullable)
// receives the total of every segment (0 for empty ones).
int32_t launch_scan_csr(int32_t dtype, const void *in, void *out, int64_t n, const int64_t *offsets,
                        int64_t nseg, void *sums, int32_t flags, void *ws, size_t ws_bytes,
                        desc_stream_t s, int cand);
size_t scan_csr_ws(int64_t n);
// Operators that only the map scan runs (the look-back scan above takes the
// value operators: sum, maximum, minimum, product, and, or, xor).
constexpr int32_t kMapScanOps = DESC_ARGMAX | DESC_ARGMIN;
// The single-pass scan through a lowered map: point g (row-major over the
// nd dims ext / stride, offset off) is in[elem(g)], its result goes to
// out[elem(g)]; segments of `period` points (nd == 0: the identity map over
// `period` points); offsets / nseg / sums: CSR segments as launch_scan_csr
// (the caller fills sums with the identity first).  Any operator flag and
// DESC_EXCLUSIVE.  Workspace: scan_contig_ws of the point count.
int32_t launch_scan_map(int32_t dtype, const void *in, void *out, int64_t off, const int64_t *ext,
                        const int64_t *stride, int nd, int64_t period, const int64_t *offsets, int64_t nseg,
                        void *sums, int32_t flags, void *ws, size_t ws_bytes, desc_stream_t s);
// The look-back scan with 4 x 4096-point tiles through a lowered map (as
// launch_scan_map, no CSR): every value operator, inclusive or exclusive;
// maps of more than two canonical dims go to launch_scan_map.  Maps of two
// dims are launched by launch_scan_mapped_2d (its own translation unit).
int32_t launch_scan_mapped(int32_t dtype, const void *in, void *out, int64_t off, const int64_t *ext,
                           const int64_t *stride, int nd, int64_t period, int32_t flags, void *ws, size_t ws_bytes,
                           desc_stream_t s);
// Arg-maximum / arg-minimum scans through a lowered map (plain or per-level
// segments): the arg look-back scan for maps of one or two canonical dims,
// launch_scan_map for others.
int32_t launch_scan_arg_mapped(int32_t dtype, const void *in, void *out, int64_t off, const int64_t *ext,
                               const int64_t *stride, int nd, int64_t period, int32_t flags, void *ws,
                               size_t ws_bytes, desc_stream_t s);
int32_t launch_scan_mapped_2d(int32_t dtype, const void *in, void *out, int64_t off, const int64_t *ext,
                              const int64_t *stride, int nd, int64_t period, int32_t flags, void *ws,
                              size_t ws_bytes, desc_stream_t s);

// Copy over a common logical domain of `nd` dims: out[ostride . p] = in[istride . p].
int32_t launch_copy_affine(const void *in, int64_t ioff, const int64_t *istride, void *out,
                           int64_t ooff, const int64_t *ostride, const int64_t *extent, int nd,
                           desc_stream_t s);
// Tiled transpose of `batch` matrices R x C (row-major, leading dim ld_in)
// into C x R (leading dim ld_out), batch strides bs_in / bs_out.
int32_t launch_transpose(const float *in, float *out, int64_t R, int64_t C, int64_t ld_in,
                         int64_t ld_out, int64_t batch, int64_t bs_in, int64_t bs_out,
                         desc_stream_t s, int cand);
int transpose_candidates();

// Schedule selection (tune.cpp): the candidate an op call should use, from
// the per-thread forced candidate, else the tuned table, else -1 (default).
int32_t schedule_for(int32_t op, int32_t dtype, int64_t n, int64_t aux);

// Matmul: FP32 SIMT (k_mm_simt.cu) and tensor-core forms (k_mm_tc.cu).
int32_t launch_sgemm(const float *A, const float *B, float *C, int64_t M, int64_t N, int64_t K, int64_t lda,
                     int64_t ldb, int64_t ldc, desc_stream_t s);
size_t mm_tc_ws(int64_t M, int64_t N, int64_t K, int planes);
// Tensor-core matmul schedule candidates: CTA pairs or not, and the
// rasterisation group in tile rows.
int mm_candidates();
void mm_candidate(int cand, int *pairs, int *group_rows, int *width);
// The schedule of a tensor-core product, decided on the host from the shape,
// the number of products, the candidate (-1: the size rule) and the number
// of CTA pairs the GPU holds at once.
struct MmPlan {
  int cand;                    // candidate taken
  int pairs;                   // 1: CTA pairs (cta_group::2), 0: single CTAs
  int width;                   // pair tiles are 256 x 256 width
  int padded;                  // an odd count of 128-row tiles padded with a zero row
  int group_rows;              // rasterisation group, in 128-row tiles
  int64_t Mp;                  // rows of the A planes the GEMM reads
  int64_t tiles_m, tiles_n;    // output tiles (tile-row pairs when pairs)
  int64_t tiles, whole;        // output tiles, and those computed whole
  int pieces;                  // K pieces of each of the other tiles
};
int32_t mm_plan(int64_t M, int64_t N, int64_t K, int nprod, int cand, int max_pairs, MmPlan *pl);
int mm_max_pairs();            // CTA pairs resident at once on the current device, 0 without one
int32_t launch_mm_tc(const float *A, int64_t a_off, int64_t a_sr, int64_t a_sc, const float *B, int64_t b_off,
                     int64_t b_sr, int64_t b_sc, float *C, int64_t M, int64_t N, int64_t K, int planes,
                     int nprod, const int *pa, const int *pb, void *ws, size_t ws_bytes, desc_stream_t s);

}  // namespace desc
