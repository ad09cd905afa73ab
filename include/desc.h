/*
 * desc.h -- C ABI of libdesc: hierarchical, view-checked data-parallel
 * primitives for one NVIDIA GB300 (sm_103a).
 *
 * The model follows Descend (Koepcke, Gorlatch, Steuwer, arXiv 2305.03448):
 * a computation is scheduled over the execution resources grid -> block ->
 * (warp ->) thread (Section 3.1), and memory is reached through *views* --
 * group, split, transpose, reverse and their map compositions -- that select
 * one part of an array per execution resource (Section 3.2).  Views never
 * move data; a chain of views is turned into one raw index (Section 5).
 *
 * Conventions shared by every entry point
 *  - Every call returns an int32 status (desc_status).  Nothing throws, aborts
 *    or traps.  All checks run before any launch; on an error nothing is
 *    launched and no output is touched.
 *  - Device buffers belong to the caller.  The library never allocates device
 *    memory in these calls: scratch space ("workspace") is passed in, sized by
 *    the matching *_workspace_size query, and must stay untouched by others
 *    until the work queued on the stream has finished.
 *  - Pointers to device data must be device (or managed) memory; a host
 *    pointer is rejected with DESC_ERR_HOST_POINTER (Section 2.3, GPU code
 *    dereferencing CPU memory).  Byte sizes are checked against the element
 *    counts the views imply (DESC_ERR_SIZE_MISMATCH; Section 2.3, a launch
 *    sized in bytes instead of elements).
 *  - Work is queued on the given stream (NULL = legacy default stream) and
 *    runs asynchronously.  Device-side failures (a bounded wait that ran out)
 *    are recorded in a per-device status word read by desc_stream_status().
 *  - Descriptors are read during the call only and never kept.
 *  - Calls are thread-safe; different streams may be used concurrently
 *    (two exceptions, stated at their declarations: desc_scan_noalloc calls
 *    must not overlap, and desc_tune_predict calls take turns).
 */
#ifndef DESC_H
#define DESC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t / CUstream. */
typedef struct CUstream_st *desc_stream_t;

typedef enum {
  DESC_OK = 0,
  DESC_ERR_INVALID_ARG = 1,     /* NULL pointer, unknown enum, negative size   */
  DESC_ERR_SHAPE = 2,           /* view type error: divisibility, split bound,
                                   select extent != resource count, selection
                                   order, rank, domain mismatch                */
  DESC_ERR_OVERLAP = 3,         /* access conflict: an element written by two
                                   threads, or written by one and read by
                                   another (Section 3.3 narrowing, Section 4) */
  DESC_ERR_HOST_POINTER = 4,    /* host memory passed where device memory is
                                   needed                                      */
  DESC_ERR_SIZE_MISMATCH = 5,   /* buffer bytes != elements * element size    */
  DESC_ERR_ALIGNMENT = 6,       /* pointer not aligned to its element size    */
  DESC_ERR_UNSUPPORTED = 7,     /* valid request this build does not handle  */
  DESC_ERR_CUDA = 8,            /* a CUDA runtime call failed                  */
  DESC_ERR_DEVICE_TIMEOUT = 9,  /* a bounded device-side wait gave up          */
  DESC_ERR_WORKSPACE = 10,      /* workspace NULL or smaller than required     */
  DESC_ERR_BARRIER = 11         /* a barrier that some thread of its scope
                                   does not reach (Section 2.2: a sync inside a
                                   split of the threads it synchronises)      */
} desc_status;

/* Execution levels (Section 3.1; the warp level is an addition: 32
 * consecutive linear thread ids, lin = x + X*(y + Y*z)). */
typedef enum {
  DESC_LEVEL_GRID = 0,
  DESC_LEVEL_BLOCK = 1,
  DESC_LEVEL_WARP = 2,
  DESC_LEVEL_THREAD = 3
} desc_level;

/* Dimensions of an execution resource (Figure "Execution Resources and
 * Dimensions").  DESC_DIM_LANE appears only in lowered maps: a THREAD select
 * that follows a WARP select binds the lane within the warp. */
typedef enum { DESC_DIM_X = 0, DESC_DIM_Y = 1, DESC_DIM_Z = 2, DESC_DIM_LANE = 3 } desc_dim;

typedef enum { DESC_I32 = 0, DESC_F32 = 1 } desc_dtype;

/* Basic views (Section 3.2 and its listing of basic view types) and select.
 *   GROUP k      [[d; n]] -> [[ [[d; k]]; n/k ]]   requires k >= 1, n % k == 0
 *   SPLIT_FST k  [[d; n]] -> [[d; k]]              requires 0 <= k <= n
 *   SPLIT_SND k  [[d; n]] -> [[d; n-k]]            element i is input i + k
 *   TRANSPOSE    [[ [[d; n]]; m ]] -> [[ [[d; m]]; n ]]
 *   REVERSE      [[d; n]] -> [[d; n]]              element i is input n-1-i
 *   SELECT       p[[e]]: the outermost dimension is distributed over the
 *                sub-resources of e along one dimension, one element each;
 *                its extent must equal their number.
 * map(v) is written as v with depth > 0: the view acts on the arrays nested
 * `depth` levels deep. */
typedef enum {
  DESC_V_GROUP = 0,
  DESC_V_SPLIT_FST = 1,
  DESC_V_SPLIT_SND = 2,
  DESC_V_TRANSPOSE = 3,
  DESC_V_REVERSE = 4,
  DESC_V_SELECT = 5
} desc_view_kind;

#define DESC_MAX_RANK 4
#define DESC_MAX_OPS 16
#define DESC_MAX_DIMS 20

typedef struct {
  int32_t kind;   /* desc_view_kind                                      */
  int32_t depth;  /* nesting depth the view acts on; must be 0 for SELECT */
  int64_t k;      /* GROUP: group size; SPLIT_*: split position; else 0  */
  int32_t level;  /* SELECT: DESC_LEVEL_BLOCK, _WARP or _THREAD           */
  int32_t dim;    /* SELECT: DESC_DIM_X, _Y or _Z (WARP and lane: X)      */
} desc_view_op;

/* A place expression: a row-major contiguous base array of `rank` extents
 * (outermost first) and the chain of views applied to it, ops[0] first. */
typedef struct {
  int32_t rank;
  int32_t nops;
  int64_t shape[DESC_MAX_RANK];
  desc_view_op ops[DESC_MAX_OPS];
} desc_view;

/* The execution resource a view is selected by: gpu.grid<grid, block>
 * (Section 3.1).  This is the *logical* resource of the view; kernels may
 * run it on fewer physical threads, each doing the work of several. */
typedef struct {
  int64_t grid[3];   /* blocks along X, Y, Z   */
  int64_t block[3];  /* threads along X, Y, Z  */
} desc_exec;

/* A lowered view: one affine map from the logical domain to the base array.
 * The logical domain is the selected dimensions, in select order, followed
 * by the dimensions left after the last view; logical point p reaches
 *     element  offset + sum_i p_i * stride_i   (in elements, row-major base).
 * level[i]/dim[i] tell which execution coordinate binds a selected
 * dimension; local dimensions have level -1 and dim -1. */
typedef struct {
  int32_t ndims;
  int32_t nsel;
  int64_t extent[DESC_MAX_DIMS];
  int64_t stride[DESC_MAX_DIMS];
  int32_t level[DESC_MAX_DIMS];
  int32_t dim[DESC_MAX_DIMS];
  int64_t offset;
  int64_t base_elems;
} desc_lowered;

/* One access of an op phase, for desc_check_disjoint.  Accesses with
 * different `buffer` ids never conflict. */
typedef struct {
  desc_lowered map;
  int32_t buffer;
  int32_t is_write;
} desc_access;

/* Human-readable name of a status code (static storage). */
const char *desc_status_string(int32_t status);

/* ABI version, (major << 16) | minor. */
int32_t desc_version(void);

/* ---- View lowering (host only, no GPU needed) ------------------------
 * Section 5: views are compiled into raw indices, transforming the index
 * view by view starting with the view applied last.  Because every basic
 * view is affine on its input index, the whole chain lowers to one affine
 * map.  Validates the view types (DESC_ERR_SHAPE) and, when `ex` is not
 * NULL, that each select's extent equals its resource count and that
 * selections narrow block -> warp -> thread (Section 3.3).  `out` is written
 * only on success. */
int32_t desc_lower_view(const desc_view *v, const desc_exec *ex, desc_lowered *out);

/* ---- Access-conflict check (host only, no GPU needed) ----------------
 * Section 3.3 (narrowing, synchronization) and Section 4
 * (access_safety_check): within one phase between barriers, no element may
 * be written by two threads, or written by one thread and read by another.
 * Each access is enumerated per thread of the grid `ex`: a thread reaches
 * the logical points whose selected coordinates equal its own; execution
 * dimensions an access does not select replicate it.  Returns DESC_OK or
 * DESC_ERR_OVERLAP; on overlap, *first_conflict (if not NULL) receives the
 * smallest conflicting element index over all buffers.
 * Uses a structural proof for affine maps (sorted strides) and exact
 * enumeration otherwise; DESC_ERR_UNSUPPORTED if enumeration would exceed
 * 2^24 (element, thread) pairs. */
int32_t desc_check_disjoint(const desc_access *acc, int32_t n, const desc_exec *ex,
                            int64_t *first_conflict);
/* The same check; *method (if not NULL) receives which checks decided the
 * buffers that have a write: DESC_DECIDED_STRUCTURAL when the structural
 * argument settled at least one of them (every element written by several
 * threads, or an injective map written by one thread each), and
 * DESC_DECIDED_ENUMERATION when at least one needed exact enumeration. */
#define DESC_DECIDED_STRUCTURAL 1
#define DESC_DECIDED_ENUMERATION 2
int32_t desc_check_disjoint_ex(const desc_access *acc, int32_t n, const desc_exec *ex,
                               int64_t *first_conflict, int32_t *method);

/* ---- Programs: accesses, barriers and splits across a kernel body ----
 * Section 3.3 and Section 4 track, per execution resource, which places
 * were accessed; a barrier releases the accesses of the threads it
 * synchronises (Section 3.3, "Synchronization"), and a barrier inside a
 * split of the threads it synchronises is rejected (Section 2.2, the
 * "barrier not allowed here" example).  desc_check_program runs these checks
 * over a whole kernel body given as a flattened statement tree:
 *   ACCESS  one view access (lowered map, buffer id, read or write) by every
 *           thread of the current (sub-)resource; its selected coordinates
 *           are relative to that sub-resource and each select's extent must
 *           equal the sub-resource's count (DESC_ERR_SHAPE otherwise);
 *   SYNC    level BLOCK (__syncthreads: releases earlier accesses between
 *           threads of the same block), WARP (__syncwarp: between threads of
 *           the same warp) or GRID (a kernel boundary: releases everything;
 *           only outside every split);
 *   SPLIT   level BLOCK (the grid's blocks along dim), THREAD (each block's
 *           threads along dim) or WARP (each block's warps, dim X): the first
 *           `n_first` statements after it run on coordinates < at, the next
 *           `n_second` on the rest (coordinates relative to `at`); the two
 *           parts run concurrently, and the statements after the split run
 *           on the whole resource again.
 * Two accesses conflict when they reach the same element of the same buffer
 * from two threads, at least one writes, and no barrier since the earlier
 * one synchronises both threads.  Returns DESC_OK; DESC_ERR_OVERLAP with
 * *bad_stmt the first conflicting access and *first_conflict its smallest
 * conflicting element; DESC_ERR_BARRIER with *bad_stmt the offending SYNC
 * (a BLOCK sync inside a THREAD or WARP split, a WARP sync inside a THREAD
 * split or in blocks whose thread count is not a multiple of 32, a GRID sync
 * inside any split); DESC_ERR_SHAPE (a split position outside (0, extent),
 * a select extent that does not match its sub-resource, warp selects where
 * the threads are split); DESC_ERR_INVALID_ARG (malformed tree);
 * DESC_ERR_UNSUPPORTED beyond 2^22 recorded (element, thread) pairs.
 * Host only; exact enumeration. */
typedef enum { DESC_STMT_ACCESS = 0, DESC_STMT_SYNC = 1, DESC_STMT_SPLIT = 2 } desc_stmt_kind;
typedef struct {
  int32_t kind;
  int32_t level;               /* SYNC / SPLIT: a desc_level                  */
  int32_t dim;                 /* SPLIT: DESC_DIM_X / Y / Z                    */
  int32_t n_first, n_second;   /* SPLIT: flattened statements of each part   */
  int64_t at;                  /* SPLIT: first part = coordinates < at        */
  desc_access access;          /* ACCESS                                      */
} desc_stmt;
int32_t desc_check_program(const desc_stmt *prog, int32_t n, const desc_exec *ex, int32_t *bad_stmt,
                           int64_t *first_conflict);

/* ---- Reduce ----------------------------------------------------------
 * Section 5 benchmark "block-wide parallel reduction"; the operator is a sum.
 * out[o] = sum of in[index(p)] over the logical points p whose selected
 * coordinates at levels <= out_level linearise (row-major, select order) to
 * o.  out_level = GRID gives one scalar.  in: base array of `v` (dtype,
 * in_bytes = elements * 4).  out: the number of outputs * 4 bytes.
 * DESC_I32 sums wrap modulo 2^32 and are bit-exact; DESC_F32 sums use FP32
 * arithmetic (error within 1e-5 * sum|x|), with compensated (Kahan)
 * accumulation when flags has DESC_KAHAN. */
#define DESC_KAHAN 1
/* Operators other than the sum (Section 5 fixes no operator; a generic
 * reduce or scan takes any associative one).  At most one operator flag:
 *   DESC_MAX / DESC_MIN      maximum / minimum, exact in both dtypes (FP32
 *                            follows IEEE maxNum / minNum: a NaN operand is
 *                            ignored unless every operand is NaN)
 *   DESC_PROD                product: int32 modulo 2^32 (exact); FP32 in FP32
 *                            arithmetic, relative error within
 *                            gamma_(m-1) = (m-1) u / (1 - (m-1) u), u = 2^-24,
 *                            for m factors when no partial product overflows
 *                            or falls below the normal range
 *   DESC_AND / DESC_OR / DESC_XOR  bitwise, int32 only (exact)
 *   DESC_ARGMAX / DESC_ARGMIN      the index, in the base array, of the
 *                            element holding the maximum / minimum value
 *                            (ties: the smallest index; FP32 NaNs lose to
 *                            every number); the output is int32 whatever the
 *                            input dtype, and the base array must have fewer
 *                            than 2^30 elements for scans, 2^31 for reduces
 * The value of an empty reduction or segment is the operator's identity: 0
 * for the sum, or and xor, INT32_MIN or -inf for the maximum, INT32_MAX or
 * +inf for the minimum, 1 for the product, all ones for and, and index -1 for
 * the arg operators.  DESC_KAHAN counts as the (compensated) sum's flag. */
#define DESC_MAX (1 << 1)
#define DESC_MIN (1 << 2)
/* Scans: out[p] combines the inputs strictly before p in its segment (the
 * identity for a segment's first point) instead of up to and including p. */
#define DESC_EXCLUSIVE (1 << 3)
#define DESC_PROD (1 << 4)
#define DESC_AND (1 << 5)
#define DESC_OR (1 << 6)
#define DESC_XOR (1 << 7)
#define DESC_ARGMAX (1 << 8)
#define DESC_ARGMIN (1 << 9)
int32_t desc_reduce_workspace_size(const desc_view *v, const desc_exec *ex, int32_t out_level,
                                   int32_t dtype, size_t *bytes);
int32_t desc_reduce(const desc_view *v, const desc_exec *ex, int32_t out_level, int32_t dtype,
                    const void *in, size_t in_bytes, void *out, size_t out_bytes, int32_t flags,
                    void *ws, size_t ws_bytes, desc_stream_t stream);

/* ---- Inclusive scan --------------------------------------------------
 * Section 5 benchmark "scan" (inclusive sum).  Segments are the logical
 * points that share their selected coordinates at levels <= seg_level
 * (GRID: one segment).  Within a segment, in logical order,
 * out[index(p)] = sum of in[index(q)] for q <= p.  `out` has the same base
 * array as `in` and is written through the same view; elements the view
 * does not reach are left untouched.  in == out (in place) is allowed.
 * DESC_I32 wraps modulo 2^32 (bit-exact); DESC_F32 has per-element error
 * within 1e-5 * sum_{q<=p} |x_q| (FP32 arithmetic, compensated carries).
 * flags: one operator flag (see desc_reduce; operators other than the sum
 * always take the default tile) and DESC_EXCLUSIVE (q < p instead of
 * q <= p).  With DESC_ARGMAX / DESC_ARGMIN, out[index(p)] is the int32 index
 * in the base array of the element chosen among the q <= p (or q < p). */
/* Test hook for the bounded waits: tile 1 never publishes, and the waits
 * give up after tens of milliseconds, so the call records
 * DESC_ERR_DEVICE_TIMEOUT (read by desc_stream_status) instead of hanging.
 * Not for production use: the output is left incomplete. */
#define DESC_DEBUG_STALL_TILE (1 << 16)
int32_t desc_scan_workspace_size(const desc_view *v, const desc_exec *ex, int32_t seg_level,
                                 int32_t dtype, size_t *bytes);
int32_t desc_scan(const desc_view *v, const desc_exec *ex, int32_t seg_level, int32_t dtype,
                  const void *in, size_t in_bytes, void *out, size_t out_bytes, int32_t flags,
                  void *ws, size_t ws_bytes, desc_stream_t stream);

/* ---- Scan without any device allocation --------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that may not allocate device memory at the time they call: for example a
 * plugin whose host framework owns and budgets every device allocation, an
 * out-of-memory or allocator callback that must not re-enter the allocator,
 * or a real-time loop that forbids allocation after start-up.  Such callers
 * cannot obtain the workspace desc_scan needs.
 *
 * desc_scan_noalloc computes what desc_scan computes (inclusive sums, no
 * flags), for views whose scan runs over one contiguous run of the base array
 * (for example the plain array, a split of it, or groups selected at
 * seg_level); other views return DESC_ERR_UNSUPPORTED.  It always runs the
 * 16384-element tile, so for int32 its results equal desc_scan's bit for bit,
 * while for FP32 they may differ from a desc_scan that runs another tile in
 * the last bits, both within the same 1e-5 * sum_{q<=p} |x_q| bound.  It takes no workspace: its scratch is a fixed
 * static device array inside the library, large enough for
 * DESC_SCAN_NOALLOC_MAX_ELEMS elements (256 bytes plus 128 bytes per 16384
 * elements, about 2 MiB).  Every GPU that loads the library holds that array
 * until the process exits.  A larger scan returns DESC_ERR_WORKSPACE and
 * launches nothing.  The call allocates nothing: no cudaMalloc, no cudaFree,
 * no allocating library routine.
 *
 * All calls on a device share the one array and the call clears what it
 * needs, so calls must not overlap on the GPU: two of them in flight at once
 * (on different streams, or from different threads) race on the scratch and
 * give wrong results.  Order them on one stream or synchronise between them.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  The
 * stream must belong to the current device. */
#define DESC_SCAN_NOALLOC_MAX_ELEMS (1LL << 28)
int32_t desc_scan_noalloc(const desc_view *v, const desc_exec *ex, int32_t seg_level, int32_t dtype,
                          const void *in, size_t in_bytes, void *out, size_t out_bytes,
                          desc_stream_t stream);

/* ---- Transpose (view-to-view copy) ----------------------------------
 * Section 1 / Section 5 benchmark "matrix transposition", generalised to any
 * pair of views with the same logical domain:
 *     out[index_out(p)] = in[index_in(p)]  for every logical point p.
 * A transpose is in_v = [R][C] with one TRANSPOSE view and out_v = [C][R].
 * Bit copy (NaN payloads kept).  `ex` may be NULL when neither view selects.
 * The output map must be injective, and when in and out are the same buffer
 * the reads and writes must not conflict (DESC_ERR_OVERLAP); partially
 * overlapping distinct buffers are rejected too. */
int32_t desc_transpose(const desc_view *in_v, const desc_view *out_v, const desc_exec *ex,
                       int32_t dtype, const void *in, size_t in_bytes, void *out, size_t out_bytes,
                       desc_stream_t stream);

/* ---- Matrix multiplication ------------------------------------------------
 * Section 5 benchmark "matrix multiplication": C = A B with FP32 A (M x K),
 * FP32 B (K x N) and FP32 C (M x N, row-major, contiguous).  a_v / b_v are
 * views of the buffers A and B whose lowered maps are 2-D, extents (M, K) and
 * (K, N), without selects (NULL: row-major contiguous); a transposed operand
 * is a TRANSPOSE view.  precision:
 *   DESC_MM_FP32_SIMT  FP32 fused multiply-adds on the CUDA cores; needs unit
 *                      stride along K for A and along N for B
 *   DESC_MM_BF16       A and B rounded to BF16 (nearest even), one tcgen05
 *                      product, FP32 accumulation in tensor memory
 *   DESC_MM_SPLIT3     x = x0 + x1 + x2 with BF16 terms (x0 = bf16(x),
 *                      x1 = bf16(x - x0), x2 = bf16(x - x0 - x1)); the six
 *                      products A_i B_j with i + j <= 2, FP32 accumulation
 *   DESC_MM_SPLIT2     two terms, the three products with i + j <= 1
 * The tensor-core forms first write the BF16 terms of A and of B transposed
 * into the workspace (zero padded to 128 / 256 / 64 multiples of M / N / K).
 * The split forms sum each half of the K range separately in FP32 and add
 * the two (on 256 x 512 output tiles the first half's sums wait in the
 * workspace, 512 KB per CTA pair the GPU holds at once); output tiles of the
 * last, partial wave may be cut along K into up to four pieces whose FP32
 * partial tiles (also in the workspace, at most 512 KB per CTA pair) are
 * added in a fixed order, so results do not vary between runs or between
 * tile shapes.  Relative Frobenius
 * error against the FP64 product (N(0,1) data, K = 8192): SPLIT3 <= 1e-5,
 * BF16 <= 1e-2.  C must not overlap A or B.  The call allocates nothing and
 * issues only kernel launches, so it can be captured in a CUDA graph; the
 * first tensor-core call or desc_matmul_workspace_size on a device sets the
 * kernels' attributes, so make one of them before capturing. */
typedef enum { DESC_MM_FP32_SIMT = 0, DESC_MM_BF16 = 1, DESC_MM_SPLIT3 = 2, DESC_MM_SPLIT2 = 3 } desc_mm_precision;
int32_t desc_matmul_workspace_size(int64_t M, int64_t N, int64_t K, int32_t precision, size_t *bytes);
int32_t desc_matmul(const desc_view *a_v, const desc_view *b_v, int64_t M, int64_t N, int64_t K, const float *A,
                    size_t a_bytes, const float *B, size_t b_bytes, float *C, size_t c_bytes, int32_t precision,
                    void *ws, size_t ws_bytes, desc_stream_t stream);

/* The schedule a tensor-core form of desc_matmul takes for a shape (host
 * only, no launch).  candidate: -1 for what desc_matmul would take (the
 * forced or tuned candidate, else the size rule), or 0 .. 5 (see
 * desc_candidate_count for DESC_OP_MATMUL).  max_pairs: the number of CTA
 * pairs the GPU holds at once; 0 asks the current device (DESC_ERR_CUDA
 * without one).  precision must be DESC_MM_BF16, DESC_MM_SPLIT2 or
 * DESC_MM_SPLIT3; M, N, K must be positive. */
typedef struct {
  int32_t candidate;    /* the schedule candidate taken */
  int32_t pairs;        /* 1: CTA pairs over 256-row tiles, 0: single CTAs over 128-row tiles */
  int32_t tile_n;       /* output tile columns: 256, or 512 for the wide pair tiles */
  int32_t padded;       /* 1: an odd count of 128-row tiles padded with a zero tile row */
  int64_t rows;         /* rows of the A terms the GEMM reads (M rounded up, padding included) */
  int64_t tiles;        /* output tiles */
  int64_t whole_tiles;  /* tiles computed whole; each of the others is cut along K into `pieces` */
  int32_t pieces;
  int32_t max_pairs;    /* the resident pair count the plan used */
} desc_mm_plan;
int32_t desc_matmul_plan(int64_t M, int64_t N, int64_t K, int32_t precision, int32_t candidate,
                         int32_t max_pairs, desc_mm_plan *plan);

/* ---- Split launch: two ops on the two parts of one grid -------------------
 * Section 3.3 splits an execution resource so that its parts run different
 * code.  desc_split_reduce_transpose runs ONE kernel launch whose first
 * blocks compute what desc_reduce computes for the view `rv` (sum; the view
 * must reduce contiguous runs longer than 4096 elements, e.g. the whole
 * array or group<k>[[block]] with k > 4096, else DESC_ERR_UNSUPPORTED) and
 * whose other blocks transpose the row-major R x C FP32 matrix tin into the
 * C x R matrix tout (what desc_transpose computes for a transpose view).
 * The four buffers must not overlap (DESC_ERR_OVERLAP): the two parts are
 * disjoint, which is what makes them safe to run concurrently.  ws: at least
 * desc_reduce_workspace_size for rv.  Results are bit-identical to the two
 * separate calls with the default schedules. */
int32_t desc_split_reduce_transpose(const desc_view *rv, const desc_exec *rex, int32_t out_level, int32_t dtype,
                                    const void *rin, size_t rin_bytes, void *rout, size_t rout_bytes, void *ws,
                                    size_t ws_bytes, const float *tin, float *tout, int64_t R, int64_t C,
                                    desc_stream_t stream);

/* ---- Segmented reduce + scan (batched) -------------------------------------
 * Many independent segments in one launch: segment s is in[offsets[s] ..
 * offsets[s+1]) of a contiguous array of `total` elements.  For every segment
 * scan_out gets its inclusive prefix sums (the Section 5 scan per segment) and
 * sums_out[s] its total (the reduce; 0 for an empty segment), both from one
 * read of the input by the look-back scan with segment heads taken from the
 * offsets.  d_offsets: device int64 array of nseg + 1 entries, nondecreasing,
 * offsets[0] = 0, offsets[nseg] = total (checked when flags has
 * DESC_CHECK_OFFSETS, which copies them to the host; unchecked bad offsets
 * give wrong values but no out-of-bounds access).  dtype DESC_I32 (wrap-around,
 * bit-exact) or DESC_F32 (per-element error within 1e-5 * sum_{q<=p} |x_q|
 * of the segment).  in == scan_out is allowed.  flags may add DESC_MAX or
 * DESC_MIN (scans and totals under that operator; an empty segment's total is
 * the operator's identity) and DESC_EXCLUSIVE (exclusive scans; the totals are
 * unchanged); any operator flag of desc_reduce may be given (arg operators:
 * scan_out and sums_out receive int32 element indices of the array, -1 for
 * an empty segment's total). */
#define DESC_CHECK_OFFSETS (1 << 17)
int32_t desc_segmented_workspace_size(int64_t nseg, int64_t total, size_t *bytes);
int32_t desc_segmented_reduce_scan(const int64_t *d_offsets, int64_t nseg, int64_t total, int32_t dtype,
                                   const void *in, void *scan_out, void *sums_out, int32_t flags, void *ws,
                                   size_t ws_bytes, desc_stream_t stream);

/* The same work as a CUDA graph, captured once and replayed: create captures
 * the launch sequence of desc_segmented_reduce_scan for fixed pointers and
 * sizes (the offsets are checked once, here); launch replays it on a stream;
 * destroy frees the graph.  The handle owns host-side graph objects only. */
typedef struct desc_graph_st *desc_graph_t;
int32_t desc_segmented_graph_create(const int64_t *d_offsets, int64_t nseg, int64_t total, int32_t dtype,
                                    const void *in, void *scan_out, void *sums_out, void *ws, size_t ws_bytes,
                                    desc_graph_t *graph);
int32_t desc_graph_launch(desc_graph_t graph, desc_stream_t stream);
int32_t desc_graph_destroy(desc_graph_t graph);

/* Baseline for the batched form: one scan launch and one reduce launch per
 * segment (h_offsets on the host), through desc_scan and desc_reduce.  Same
 * results; exists to measure what batching saves.  ws: at least
 * desc_segmented_workspace_size bytes. */
int32_t desc_segmented_reduce_scan_per_segment(const int64_t *h_offsets, int64_t nseg, int32_t dtype,
                                               const void *in, void *scan_out, void *sums_out, void *ws,
                                               size_t ws_bytes, desc_stream_t stream);

/* ---- Schedules: candidates, exhaustive tuner, learned picker ---------------
 * Not in the paper.  Each tunable op has a few compiled schedule candidates
 * (candidate 0 is the default):
 *   DESC_OP_REDUCE     chunked reduce: (vectors in flight per thread, target
 *                      CTA count, load path) in {(8,1216,s), (4,1216,s),
 *                      (8,608,s), (4,2432,s), (8,2432,s), (8,304,s),
 *                      (4,2432,r), (8,1216,r)}; s = evict-first streaming
 *                      loads, r = read-only path without L1 allocation
 *   DESC_OP_SCAN       look-back scan: tile of 4096 x {4, 2, 1} elements
 *   DESC_OP_TRANSPOSE  tiles of {64, 32} squared
 *   DESC_OP_SEGMENTED  CSR look-back scan: tile of 4096 x {4, 2, 1} elements;
 *                      or one warp (3), or one CTA of 256 threads (4), per
 *                      segment, walking it in steps of 4 points per thread
 *   DESC_OP_MATMUL     tensor-core forms: {CTA pairs on 256 x 256 tiles where
 *                      the 128-row tiles pair up, one CTA per 128 x 256 tile}
 *                      x {wide, narrow} rasterisation groups: 16 / 4 tile
 *                      rows (single) and 8 / 2 tile-row pairs (pairs); and
 *                      pairs on 256 x 512 tiles, wide / narrow groups
 * Ops look up the candidate recorded for their bucket -- (GPU model, op,
 * dtype, floor(log2 n), floor(log2(aux + 1))) with n and aux as the op call
 * sees them (below) -- in a process-wide table (thread-safe), else use
 * candidate 0.  A table saved on one GPU model is not used on another. */
typedef enum {
  DESC_OP_REDUCE = 0,
  DESC_OP_SCAN = 1,
  DESC_OP_TRANSPOSE = 2,
  DESC_OP_SEGMENTED = 3,
  DESC_OP_MATMUL = 4
} desc_op;
#define DESC_NUM_FEATURES 40
/* One call's shape.  With `view` NULL the call is the op's plain form: reduce
 * of n elements (aux > 1: n / aux elements per output, selected per block),
 * scan of n elements, transpose of an aux x (n / aux) matrix, segmented with
 * aux segments of n elements in all, matmul M = n, N = aux, K = k.  With a
 * view (reduce and scan only), the call is desc_reduce / desc_scan through
 * that view, the execution resource `ex` and the level `level` (out_level /
 * seg_level); n and aux are then taken from the lowered view: n = the points
 * reduced or scanned, aux = the outputs (reduce) or segments (scan) when more
 * than one, else 0.  seg_lengths (segmented): the aux segment lengths on the
 * host, read during the call only; NULL leaves the length histogram zero. */
typedef struct {
  int32_t op;                  /* desc_op                                                   */
  int32_t dtype;               /* DESC_I32 / DESC_F32 (matmul: DESC_F32)                     */
  int64_t n;                   /* elements; matmul: M                                       */
  int64_t aux;                 /* reduce: outputs; transpose: rows; segmented: segments;
                                  scan: 0; matmul: N                                         */
  int64_t k;                   /* matmul: K; other ops: 0                                   */
  const int64_t *seg_lengths;  /* segmented: aux lengths (host), or NULL                    */
  const desc_view *view;       /* reduce / scan: the call's view, or NULL                   */
  const desc_exec *ex;         /* the view's execution resource (NULL without selects)      */
  int32_t level;               /* reduce: out_level; scan: seg_level (with a view)           */
} desc_problem;
/* Device buffers a measurement runs on (the caller owns them): in (the input:
 * n elements of dtype, or the view's base array; matmul: A, M x K FP32), out
 * (reduce: the outputs; matmul: M x N; others: as many elements as in), sums
 * (segmented: aux), offsets (segmented: aux + 1, device int64), ws (at least
 * the op's workspace), in2 (matmul: B, K x N FP32; else unused).  Matmul
 * problems are timed in DESC_MM_BF16. */
typedef struct {
  const void *in;
  void *out;
  void *sums;
  const int64_t *offsets;
  void *ws;
  size_t ws_bytes;
  const void *in2;
} desc_tune_buffers;

int32_t desc_candidate_count(int32_t op, int32_t *count);
/* Features of (problem, candidate) for the cost model, DESC_NUM_FEATURES
 * floats:
 *   [0, 5)   op one-hot            [5, 7)   dtype one-hot (I32, F32)
 *   [7]      log2 n / 32           [8]      log2(aux + 1) / 32
 *   [9]      log2(n / (aux + 1) + 1) / 32
 *   [10, 18) segmented: fraction of segments with floor(log2 len) in [0, 3),
 *            [3, 6), ..., [21, 24) (empty segments in the first bucket),
 *            computed here from seg_lengths
 *   [18]     log2 of the candidate's tile elements / 32
 *   [19]     vectors in flight / 16   [20] log2 CTA target or group / 16
 *   [21, 29) candidate index one-hot  [29] load path   [30] log2(K + 1) / 32
 *   [31]     CTA pairs
 *   [32, 37) view composition: number of group, split (fst or snd),
 *            transpose, reverse and select views, each / 8
 *   [37]     the deepest nesting a view acts on (map depth) / 4
 *   [38]     1 when the lowered map takes the op's hand-indexed kernel
 *            (contiguous runs, or a tiled 2-D transposition), else 0
 *   [39]     dims of the lowered map after merging neighbours / 8 */
int32_t desc_features(const desc_problem *p, int32_t cand, float *out, int32_t nout);
/* Times every candidate on the given buffers (reps launches each, CUDA events
 * on the stream, median), writing microseconds to us[count].  Synchronises. */
int32_t desc_tune_measure(const desc_problem *p, const desc_tune_buffers *b, int32_t reps, desc_stream_t stream,
                          float *us);
/* Times the ncand candidates listed in cands (each reps launches, median), in
 * rounds that visit every listed candidate once before the next round (so slow
 * drifts of the clock touch all of them alike); us[i] belongs to cands[i]. */
int32_t desc_tune_measure_cands(const desc_problem *p, const desc_tune_buffers *b, const int32_t *cands,
                                int32_t ncand, int32_t reps, desc_stream_t stream, float *us);
/* Exhaustive autotuning: measure all candidates, record the fastest (ties:
 * the lowest index) for the problem's bucket, return it. */
int32_t desc_tune_exhaustive(const desc_problem *p, const desc_tune_buffers *b, int32_t reps,
                             desc_stream_t stream, int32_t *best);
/* Table entries for the current device's GPU model (no GPU: the model name
 * "none"). */
int32_t desc_tune_record(const desc_problem *p, int32_t cand);
int32_t desc_tune_lookup(const desc_problem *p, int32_t *cand);   /* -1 when nothing is recorded */
int32_t desc_tune_clear(void);
/* Text file, one bucket per line: GPU model (spaces as '_'), op, dtype,
 * log2 n, log2(aux + 1), candidate.  Loading merges the file into the table. */
int32_t desc_tune_save(const char *path);
int32_t desc_tune_load(const char *path);
/* Per-thread override used while measuring: ops of `op` use candidate `cand`
 * (-1: back to the table). */
int32_t desc_force_candidate(int32_t op, int32_t cand);

/* ---- View-overhead switch --------------------------------------------
 * Section 5 compares kernels whose indexing comes from views with
 * hand-indexed CUDA of the same operations.  Here every view is lowered to
 * an affine map; where that map has a simple form (contiguous runs, a 2-D
 * transposition) a hand-indexed kernel runs, and otherwise a general kernel
 * evaluates the map element by element.  With `on` != 0 the calling thread's
 * desc_reduce, desc_scan and desc_transpose calls (and their workspace
 * queries) take the general path even where a hand-indexed kernel applies:
 * reduce through the affine reduction kernel, scan through an affine gather
 * into the workspace, the scan and an affine scatter, transpose through the
 * affine copy kernel.  Results are the same; only the time differs.  Query
 * the workspace with the same setting as the call.  Returns DESC_OK. */
int32_t desc_force_generic(int32_t on);

/* ---- Cost model: 3-layer MLP on the GPU ------------------------------------
 * y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 predicts log(time in us) of a
 * (problem, candidate) feature row; loss = mean squared error.  Parameters are
 * one FP32 device vector [W1 (H x F, row-major), b1, W2 (H x H), b2, w3, b3]
 * (desc_mlp_param_count), owned by the caller, as are the Adam moments m and v
 * (same length) and the workspace.  F <= 64, H <= 64 (H a multiple of 32).
 * Forward, backward and Adam run in this library's kernels. */
int32_t desc_mlp_param_count(int32_t F, int32_t H, int64_t *count);
int32_t desc_mlp_workspace_size(int32_t F, int32_t H, int64_t rows, size_t *bytes);
int32_t desc_mlp_forward(const float *params, int32_t F, int32_t H, const float *X, int64_t rows, float *y,
                         void *ws, size_t ws_bytes, desc_stream_t stream);
/* grad = d loss / d params over the rows (mean squared error against t). */
int32_t desc_mlp_backward(const float *params, int32_t F, int32_t H, const float *X, const float *t, int64_t rows,
                          float *grad, void *ws, size_t ws_bytes, desc_stream_t stream);
/* One Adam step (Kingma and Ba, Algorithm 1; step counts from 1). */
int32_t desc_mlp_adam(float *params, const float *grad, float *m, float *v, int64_t count, int32_t step, float lr,
                      float beta1, float beta2, float eps, desc_stream_t stream);
/* Minibatch training: epochs over rows (taken in the given order, batches of
 * `batch` consecutive rows); *loss receives the mean loss of the last epoch. */
int32_t desc_mlp_train(float *params, float *grad, float *m, float *v, int32_t F, int32_t H, const float *X,
                       const float *t, int64_t rows, int32_t epochs, int32_t batch, float lr, void *ws,
                       size_t ws_bytes, desc_stream_t stream, float *loss);
/* Scores ncand feature rows (device) and writes the index of the smallest
 * prediction (ties: the lowest) to *best (device int32) and all predictions
 * to pred (device, ncand). */
int32_t desc_mlp_pick(const float *params, int32_t F, int32_t H, const float *Xcand, int32_t ncand, float *pred,
                      int32_t *best, desc_stream_t stream);
/* Learned schedules: the model (kept by reference: the caller keeps params
 * alive and unchanged while it is set) picks the candidate of a problem
 * without timing, and the pick is recorded like a tuned one.
 * desc_tune_predict stages the candidates' features in device memory the
 * library owns, runs the pick kernel on `stream` and waits for it: calls from
 * several threads are serialised by a library-wide lock (each gets its own
 * pick), the call synchronises the stream, and it cannot be captured into a
 * CUDA graph. */
int32_t desc_tune_set_model(const float *params, int32_t F, int32_t H);
int32_t desc_tune_predict(const desc_problem *p, desc_stream_t stream, int32_t *best);

/* Per-device status word: waits for the stream, returns the first device
 * error recorded since the last call (DESC_OK if none) and clears it. */
int32_t desc_stream_status(desc_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* DESC_H */
