// Reduce kernels (sum over a lowered view).
//
// Three schedules, picked on the host from the lowered map:
//  * runs:   every output sums one contiguous run of `len` elements, runs
//            starting at start + o * seg_stride.  Long runs are cut into
//            chunks, one CTA per (run, chunk); the chunks interleave in
//            stripes of UNROLL x 256 vectors (all CTAs of a run sweep the run
//            together), read with 128-bit loads, UNROLL vectors in flight per
//            thread,
//            merges warp-wide with shuffles and block-wide through shared
//            memory; the last CTA of a run (atomic ticket) merges the chunk
//            partials in chunk order.  Short runs go one warp or one thread
//            per output.
//  * affine: any other map; same chunk/partial structure, with every element
//            index decoded from the remaining dims.
// int32 sums wrap mod 2^32 (any order gives the same bits); FP32 sums are
// plain or compensated (Neumaier) FP32.  Other operators (maximum, minimum,
// product, bitwise and / or / xor, arg-maximum / arg-minimum) run through
// the same kernels with their accumulator; the arg accumulators also take
// each element's index in the base array and write that index (int32).
#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "k_bodies.cuh"
#include "k_common.cuh"

namespace desc {
namespace {

constexpr int kThreads = 256;
constexpr int64_t kSmallRun = 16;          // <= this: one thread per output
constexpr int64_t kWarpRun = 4096;         // <= this: one warp per output

// Schedule candidates of the chunked kernel (candidates.h).
using Cand = ReduceCand;
constexpr const Cand *kCands = kReduceCands;
constexpr int kNumCands = kNumReduceCands;

// A candidate's CTA target counts whole waves where the kernel holds 8 CTAs
// on each SM (1216 = 8 x 152).  A kernel that holds fewer (the arg
// accumulators at 8 vectors in flight take 40 registers: 6 a SM) would leave
// a ragged last wave, so a target above one wave of the kernel's own
// (per_wave = CTAs a SM x SMs) is cut to whole waves; a target within one
// wave is kept.  Targets only shrink, so no candidate makes more chunks than
// max_chunks sized the workspace for.
int64_t chunks_for(int64_t len, int64_t nout, const Cand &c, int64_t per_wave = 0) {
  const int64_t per_cta_min = int64_t(kThreads) * 4 * c.unroll;
  const int64_t target = per_wave > 0 && c.target_ctas > per_wave ? (c.target_ctas / per_wave) * per_wave
                                                                    : c.target_ctas;
  int64_t by_fill = (target + nout - 1) / std::max<int64_t>(nout, 1);
  int64_t by_len = (len + per_cta_min - 1) / per_cta_min;
  return std::max<int64_t>(1, std::min(by_fill, by_len));
}

// The most chunks any candidate uses (sizes the partials).
int64_t max_chunks(int64_t len, int64_t nout) {
  int64_t m = 1;
  for (int i = 0; i < kNumCands; ++i) m = std::max(m, chunks_for(len, nout, kCands[i]));
  return m;
}

template <class A>
__device__ __forceinline__ float final_value(const A &a);
template <>
__device__ __forceinline__ float final_value(const AccF32 &a) { return a.s; }
template <>
__device__ __forceinline__ float final_value(const AccKahan &a) { return __fadd_rn(a.s, a.c); }

template <class A>
struct IsArg : std::false_type {};
template <class T, bool MAX>
struct IsArg<AccArg<T, MAX>> : std::true_type {};
template <class A>
struct IsPlainValue : std::false_type {};   // accumulators that hold the result in .v
template <class T, bool MAX>
struct IsPlainValue<AccExt<T, MAX>> : std::true_type {};
template <class T>
struct IsPlainValue<AccProd<T>> : std::true_type {};
template <int OP>
struct IsPlainValue<AccBits<OP>> : std::true_type {};

template <class A, class T>
__device__ __forceinline__ void store_out(T *out, int64_t o, const A &a) {
  if constexpr (IsArg<A>::value)
    reinterpret_cast<int32_t *>(out)[o] = a.i;          // the winner's element index
  else if constexpr (IsPlainValue<A>::value)
    out[o] = __builtin_bit_cast(T, a.v);
  else
    out[o] = final_value(a);
}
template <>
__device__ __forceinline__ void store_out<AccI32, int32_t>(int32_t *out, int64_t o, const AccI32 &a) {
  out[o] = (int32_t)a.s;
}

// After a CTA has its block partial in thread 0: write it, or take part in
// the last-CTA merge of the run's partials.
template <class A, class T>
__device__ __forceinline__ void finish_chunk(A &a, A *sh, int64_t o, int64_t c, int64_t chunks,
                                             T *out, uint2 *partials, unsigned *counters) {
  if (chunks == 1) {
    if (threadIdx.x == 0) store_out<A, T>(out, o, a);
    return;
  }
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[o * chunks + c] = a.pack();
    __threadfence();
    const unsigned t = atomicAdd(&counters[o], 1u);
    last = (t == (unsigned)(chunks - 1));
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  A b;
  b.init();
  // chunk order within each thread, then a fixed tree: deterministic
  for (int64_t i = threadIdx.x; i < chunks; i += kThreads) {
    A p;
    p.unpack(__ldcg(&partials[o * chunks + i]));
    b.merge(p);
  }
  __syncthreads();
  block_merge<A, kThreads>(b, sh);
  if (threadIdx.x == 0) {
    store_out<A, T>(out, o, b);
    counters[o] = 0u;
  }
}

template <class T> struct Vec;
template <> struct Vec<int32_t> { using type = int4; };
template <> struct Vec<float> { using type = float4; };

__device__ __forceinline__ int4 ld_nc(const int4 *p) {
  int4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ float4 ld_nc(const float4 *p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}
template <int NC, class V>
__device__ __forceinline__ V ld_vec(const V *p) {
  if (NC) return ld_nc(p);
  return ld_stream(p);
}

// The work of CTA `blk` of the chunked reduce: run blk / chunks, chunk
// blk % chunks.
template <class A, class T, int kUnroll, int NC>
__device__ __forceinline__ void reduce_runs_block(const T *__restrict__ in, int64_t start, int64_t seg_stride,
                                                  int64_t len, int64_t chunks, T *__restrict__ out,
                                                  uint2 *partials, unsigned *counters, int64_t blk) {
  using V = typename Vec<T>::type;
  __shared__ A sh[kThreads / 32];
  const int64_t o = blk / chunks, c = blk % chunks;
  const int64_t e0 = start + o * seg_stride;            // element index of the run's first element
  const T *p = in + e0;
  const int64_t mis = (reinterpret_cast<uintptr_t>(p) & 15) / sizeof(T);
  const int64_t head = std::min<int64_t>(len, mis ? 4 - mis : 0);
  const int64_t nvec = (len - head) / 4;
  const int64_t tail = len - head - 4 * nvec;
  A a;
  a.init();
  const V *pv = reinterpret_cast<const V *>(p + head);
  const int64_t ev = e0 + head;                        // element index of vector 0
  // The run's vectors in stripes of kUnroll x kThreads; CTA c takes stripes
  // c, c + chunks, ... so that the CTAs of a run read neighbouring stripes
  // at the same time (DRAM rows stay open across the GPU) rather than each
  // walking a distant chunk of its own.
  constexpr int64_t kStripe = int64_t(kUnroll) * kThreads;
  const int64_t step = chunks * kStripe;
  int64_t b = c * kStripe;
  for (; b + kStripe <= nvec; b += step) {
    V x[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) x[u] = ld_vec<NC>(pv + b + u * kThreads + threadIdx.x);
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) acc_add4(a, x[u], ev + 4 * (b + u * kThreads + threadIdx.x));
  }
  if (b < nvec)                                        // the last, partial stripe
    for (int64_t i = b + threadIdx.x; i < nvec; i += kThreads) acc_add4(a, ld_vec<NC>(pv + i), ev + 4 * i);
  if (c == 0 && threadIdx.x < head) acc_add1(a, p[threadIdx.x], e0 + threadIdx.x);
  if (c == chunks - 1 && threadIdx.x < tail)
    acc_add1(a, p[head + 4 * nvec + threadIdx.x], e0 + head + 4 * nvec + threadIdx.x);
  block_merge<A, kThreads>(a, sh);
  finish_chunk<A, T>(a, sh, o, c, chunks, out, partials, counters);
}

// One CTA per (run, chunk).  grid.x = nout * chunks.
template <class A, class T, int kUnroll, int NC>
__global__ void __launch_bounds__(kThreads) reduce_runs_kernel(
    const T *__restrict__ in, int64_t start, int64_t seg_stride, int64_t len, int64_t chunks,
    int64_t /*chunk_vec*/, T *__restrict__ out, uint2 *partials, unsigned *counters) {
  reduce_runs_block<A, T, kUnroll, NC>(in, start, seg_stride, len, chunks, out, partials, counters, blockIdx.x);
}

// A split launch (Section 3.3: the parts of a split resource run different
// code): blocks [0, nred) reduce runs as reduce_runs_kernel, the others
// transpose a matrix in 64 x 64 tiles as transpose_kernel (256 threads seen
// as 32 x 8).  Each block runs one part entirely, so the barriers inside each
// part are reached by all of its threads.
struct SplitTranspose {
  const float *in;
  float *out;
  int64_t R, C, gx;
};
template <class A, class T>
__global__ void __launch_bounds__(kThreads) split_reduce_transpose_kernel(
    const T *__restrict__ in, int64_t start, int64_t seg_stride, int64_t len, int64_t chunks, T *__restrict__ out,
    uint2 *partials, unsigned *counters, int64_t nred, SplitTranspose tr) {
  __shared__ float tile[64][65];
  if (int64_t(blockIdx.x) < nred) {
    reduce_runs_block<A, T, 8, 0>(in, start, seg_stride, len, chunks, out, partials, counters, blockIdx.x);
  } else {
    const int64_t t = int64_t(blockIdx.x) - nred;
    transpose_tile<64, 8>(tr.in, tr.out, tr.R, tr.C, tr.C, tr.R, 0, 0, t % tr.gx, t / tr.gx, 0,
                          threadIdx.x & 31, threadIdx.x >> 5, tile);
  }
}

// GROUP threads per output (GROUP = 1 or 32), grid-stride over outputs.
template <class A, class T, int GROUP>
__global__ void __launch_bounds__(kThreads) reduce_short_kernel(
    const T *__restrict__ in, int64_t start, int64_t seg_stride, int64_t len, int64_t nout,
    T *__restrict__ out) {
  const int64_t gid = int64_t(blockIdx.x) * kThreads + threadIdx.x;
  const int64_t ngroups = int64_t(gridDim.x) * (kThreads / GROUP);
  const int lane = threadIdx.x % GROUP;
  for (int64_t o = gid / GROUP; o < nout; o += ngroups) {
    const int64_t e0 = start + o * seg_stride;
    const T *p = in + e0;
    A a;
    a.init();
    for (int64_t j = lane; j < len; j += GROUP) acc_add1(a, p[j], e0 + j);
    if (GROUP == 32) warp_merge(a);
    if (lane == 0) store_out<A, T>(out, o, a);
  }
}

struct AffineArgs {
  int32_t nkeep, nrest;
  int64_t keep_ext[DESC_MAX_DIMS], keep_st[DESC_MAX_DIMS];
  int64_t rest_ext[DESC_MAX_DIMS], rest_st[DESC_MAX_DIMS];
  FastDiv rest_div[DESC_MAX_DIMS];   // FAST: the summed extents as 32-bit invariant divisors
  int64_t offset, n_rest;
};

// One CTA per (output, chunk) over an arbitrary affine map; each point's
// element is decoded from its row-major index over the summed dims.  FAST
// (fewer than 2^32 summed points, extents <= 2^31): 32-bit decoding by
// multiply-high; otherwise 64-bit division.
// VEC (with FAST): the innermost summed dim is contiguous, its extent, the
// other strides and the offset are multiples of 4 and `in` is 16-byte
// aligned, so points go in groups of 4 with one 128-bit load each.
template <class A, class T, bool FAST, bool VEC>
__global__ void __launch_bounds__(kThreads) reduce_affine_kernel(
    const T *__restrict__ in, const AffineArgs args, int64_t chunks, int64_t chunk_len,
    T *__restrict__ out, uint2 *partials, unsigned *counters) {
  __shared__ A sh[kThreads / 32];
  const int64_t o = blockIdx.x / chunks, c = blockIdx.x % chunks;
  int64_t base = args.offset, r = o;
  for (int d = args.nkeep - 1; d >= 0; --d) {
    base += (r % args.keep_ext[d]) * args.keep_st[d];
    r /= args.keep_ext[d];
  }
  A a;
  a.init();
  const int64_t q1 = std::min<int64_t>(args.n_rest, (c + 1) * chunk_len);
  if (VEC) {
    // stripes of 4 x U x kThreads points; CTA c takes stripes c, c + chunks,
    // ... (the CTAs of an output sweep its points together)
    using V4 = typename std::conditional<std::is_same<T, float>::value, float4, int4>::type;
    constexpr int U = 4;                               // groups in flight per thread
    constexpr int64_t kStripe = int64_t(4) * U * kThreads;
    const int64_t qend = args.n_rest;
    for (int64_t s0 = c * kStripe; s0 < qend; s0 += chunks * kStripe) {
      const int64_t q0 = s0 + 4 * threadIdx.x;
      V4 v[U];
      int64_t ei[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t q = q0 + int64_t(u) * 4 * kThreads;
        ei[u] = 0;
        if (q < qend) {
          int64_t e = base;
          uint32_t t = (uint32_t)q;
          for (int d = args.nrest - 1; d > 0; --d) {
            const uint32_t qd = fast_div(t, args.rest_div[d]);
            e += int64_t(t - qd * args.rest_div[d].d) * args.rest_st[d];
            t = qd;
          }
          e += int64_t(t) * args.rest_st[0];
          ei[u] = e;
          v[u] = __ldcs(reinterpret_cast<const V4 *>(in + e));
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (q0 + int64_t(u) * 4 * kThreads < qend) acc_add4(a, v[u], ei[u]);
    }
  } else
  for (int64_t q = c * chunk_len + threadIdx.x; q < q1; q += kThreads) {
    int64_t e = base;
    if (FAST) {
      uint32_t t = (uint32_t)q;
      for (int d = args.nrest - 1; d > 0; --d) {
        const uint32_t qd = fast_div(t, args.rest_div[d]);
        e += int64_t(t - qd * args.rest_div[d].d) * args.rest_st[d];
        t = qd;
      }
      e += int64_t(t) * args.rest_st[0];
    } else {
      int64_t t = q;
      for (int d = args.nrest - 1; d >= 0; --d) {
        e += (t % args.rest_ext[d]) * args.rest_st[d];
        t /= args.rest_ext[d];
      }
    }
    acc_add1(a, in[e], e);
  }
  block_merge<A, kThreads>(a, sh);
  finish_chunk<A, T>(a, sh, o, c, chunks, out, partials, counters);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// CTAs of `kernel` (kThreads threads, no dynamic shared memory) that all
// SMs of the current device hold at once, asked once per kernel and device.
cudaError_t wave_ctas(const void *kernel, int64_t *out) {
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, int64_t> known;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto it = known.find({kernel, dev});
  if (it != known.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  int r = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, kernel, kThreads, 0);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  known[{kernel, dev}] = int64_t(r) * sms;
  *out = int64_t(r) * sms;
  return cudaSuccess;
}

size_t ws_for(int64_t len, int64_t nout) {
  if (len <= kWarpRun) return 0;
  const int64_t ch = max_chunks(len, nout);
  if (ch == 1) return 0;
  return align256(size_t(nout) * ch * sizeof(uint2)) + align256(size_t(nout) * sizeof(unsigned));
}

template <class A, class T>
int32_t run_runs(const T *in, int64_t start, int64_t seg_stride, int64_t len, int64_t nout, T *out,
                 void *ws, size_t ws_bytes, cudaStream_t s, int cand) {
  if (len <= kSmallRun) {
    const int64_t ctas = std::min<int64_t>((nout + kThreads - 1) / kThreads, int64_t(1) << 20);
    reduce_short_kernel<A, T, 1><<<(unsigned)ctas, kThreads, 0, s>>>(in, start, seg_stride, len, nout, out);
  } else if (len <= kWarpRun) {
    const int64_t ctas = std::min<int64_t>((nout * 32 + kThreads - 1) / kThreads, int64_t(1) << 20);
    reduce_short_kernel<A, T, 32><<<(unsigned)ctas, kThreads, 0, s>>>(in, start, seg_stride, len, nout, out);
  } else {
    const Cand &cd = kCands[(cand >= 0 && cand < kNumCands) ? cand : 0];
    auto kern = cd.unroll == 4 ? (cd.nc ? reduce_runs_kernel<A, T, 4, 1> : reduce_runs_kernel<A, T, 4, 0>)
                               : (cd.nc ? reduce_runs_kernel<A, T, 8, 1> : reduce_runs_kernel<A, T, 8, 0>);
    int64_t per_wave = 0;
    DESC_CUDA_TRY(wave_ctas(reinterpret_cast<const void *>(kern), &per_wave));
    const int64_t chunks = chunks_for(len, nout, cd, per_wave);
    uint2 *partials = nullptr;
    unsigned *counters = nullptr;
    if (chunks > 1) {
      if (!ws || ws_bytes < ws_for(len, nout)) return DESC_ERR_WORKSPACE;
      partials = static_cast<uint2 *>(ws);
      counters = reinterpret_cast<unsigned *>(static_cast<char *>(ws) +
                                              align256(size_t(nout) * max_chunks(len, nout) * sizeof(uint2)));
      DESC_CUDA_TRY(cudaMemsetAsync(counters, 0, size_t(nout) * sizeof(unsigned), s));
    }
    const int64_t nvec = len / 4 + 1;
    const int64_t chunk_vec = (nvec + chunks - 1) / chunks;
    if (nout * chunks >= (int64_t(1) << 31)) return DESC_ERR_UNSUPPORTED;
    const unsigned grid = (unsigned)(nout * chunks);
    kern<<<grid, kThreads, 0, s>>>(in, start, seg_stride, len, chunks, chunk_vec, out, partials, counters);
  }
  DESC_CUDA_TRY(cudaGetLastError());
  return DESC_OK;
}

template <class A, class T>
int32_t run_affine(const T *in, const Plan &p, T *out, void *ws, size_t ws_bytes, cudaStream_t s) {
  AffineArgs a;
  a.nkeep = p.nkeep;
  for (int i = 0; i < p.nkeep; ++i) { a.keep_ext[i] = p.keep[i].extent; a.keep_st[i] = p.keep[i].stride; }
  for (int i = 0; i < p.nrest; ++i) { a.rest_ext[i] = p.rest[i].extent; a.rest_st[i] = p.rest[i].stride; }
  int64_t *sets[1] = {a.rest_st};
  a.nrest = canon_dims(p.nrest, a.rest_ext, sets, 1);
  if (a.nrest == 0) {                                  // one point per output
    a.nrest = 1;
    a.rest_ext[0] = 1;
    a.rest_st[0] = 0;
  }
  bool fast = p.n_rest < (int64_t(1) << 32);
  for (int i = 0; i < a.nrest; ++i) {
    fast = fast && a.rest_ext[i] <= (int64_t(1) << 31);
    if (fast) a.rest_div[i] = make_fastdiv((uint32_t)a.rest_ext[i]);
  }
  a.offset = p.offset;
  a.n_rest = p.n_rest;
  const int64_t nout = p.n_keep;
  const int64_t chunks = p.n_rest <= kWarpRun ? 1 : chunks_for(p.n_rest, nout, kCands[0]);
  bool vec = fast && a.rest_st[a.nrest - 1] == 1 && a.rest_ext[a.nrest - 1] % 4 == 0 && a.offset % 4 == 0 &&
             (reinterpret_cast<uintptr_t>(in) & 15) == 0;
  for (int i = 0; i + 1 < a.nrest; ++i) vec = vec && a.rest_st[i] % 4 == 0;
  for (int i = 0; i < a.nkeep; ++i) vec = vec && a.keep_st[i] % 4 == 0;
  int64_t chunk_len = (p.n_rest + chunks - 1) / chunks;
  if (vec) chunk_len = (chunk_len + 3) / 4 * 4;        // chunks start on a group of 4
  uint2 *partials = nullptr;
  unsigned *counters = nullptr;
  if (chunks > 1) {
    if (!ws || ws_bytes < ws_for(p.n_rest, nout)) return DESC_ERR_WORKSPACE;
    partials = static_cast<uint2 *>(ws);
    counters = reinterpret_cast<unsigned *>(static_cast<char *>(ws) +
                                            align256(size_t(nout) * max_chunks(p.n_rest, nout) * sizeof(uint2)));
    DESC_CUDA_TRY(cudaMemsetAsync(counters, 0, size_t(nout) * sizeof(unsigned), s));
  }
  if (nout * chunks >= (int64_t(1) << 31)) return DESC_ERR_UNSUPPORTED;
  const unsigned grid = (unsigned)(nout * chunks);
  if (vec)
    reduce_affine_kernel<A, T, true, true><<<grid, kThreads, 0, s>>>(in, a, chunks, chunk_len, out, partials,
                                                                     counters);
  else if (fast)
    reduce_affine_kernel<A, T, true, false><<<grid, kThreads, 0, s>>>(in, a, chunks, chunk_len, out, partials,
                                                                      counters);
  else
    reduce_affine_kernel<A, T, false, false><<<grid, kThreads, 0, s>>>(in, a, chunks, chunk_len, out, partials,
                                                                       counters);
  DESC_CUDA_TRY(cudaGetLastError());
  return DESC_OK;
}

}  // namespace

size_t reduce_segments_ws(int32_t /*dtype*/, int64_t len, int64_t nout) { return ws_for(len, nout); }

int reduce_candidates() { return kNumCands; }

namespace {
template <class A, class T>
struct AccTag {
  using Acc = A;
  using Elem = T;
};

// Calls f(AccTag<accumulator, element type>{}) for the operator in `flags`
// (at most one operator flag; none: the sum, DESC_KAHAN: the compensated sum).
template <class F>
int32_t with_accumulator(int32_t dtype, int32_t flags, F &&f) {
  const int32_t op = flags & kOperatorFlags;
  if (dtype == DESC_I32) {
    switch (op) {
      case DESC_MAX: return f(AccTag<AccExt<int32_t, true>, int32_t>{});
      case DESC_MIN: return f(AccTag<AccExt<int32_t, false>, int32_t>{});
      case DESC_PROD: return f(AccTag<AccProd<int32_t>, int32_t>{});
      case DESC_AND: return f(AccTag<AccBits<0>, int32_t>{});
      case DESC_OR: return f(AccTag<AccBits<1>, int32_t>{});
      case DESC_XOR: return f(AccTag<AccBits<2>, int32_t>{});
      case DESC_ARGMAX: return f(AccTag<AccArg<int32_t, true>, int32_t>{});
      case DESC_ARGMIN: return f(AccTag<AccArg<int32_t, false>, int32_t>{});
      case 0:
      case DESC_KAHAN: return f(AccTag<AccI32, int32_t>{});   // int32 sums are exact
      default: return DESC_ERR_INVALID_ARG;
    }
  }
  switch (op) {
    case DESC_MAX: return f(AccTag<AccExt<float, true>, float>{});
    case DESC_MIN: return f(AccTag<AccExt<float, false>, float>{});
    case DESC_PROD: return f(AccTag<AccProd<float>, float>{});
    case DESC_ARGMAX: return f(AccTag<AccArg<float, true>, float>{});
    case DESC_ARGMIN: return f(AccTag<AccArg<float, false>, float>{});
    case DESC_KAHAN: return f(AccTag<AccKahan, float>{});
    case 0: return f(AccTag<AccF32, float>{});
    default: return DESC_ERR_INVALID_ARG;
  }
}
}  // namespace

int32_t launch_reduce_segments(int32_t dtype, const void *in, int64_t start, int64_t seg_stride,
                               int64_t len, int64_t nout, void *out, int32_t flags, void *ws,
                               size_t ws_bytes, desc_stream_t st, int cand) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  return with_accumulator(dtype, flags, [&](auto tag) {
    using A = typename decltype(tag)::Acc;
    using T = typename decltype(tag)::Elem;
    return run_runs<A, T>(static_cast<const T *>(in), start, seg_stride, len, nout, static_cast<T *>(out), ws,
                          ws_bytes, s, cand);
  });
}

size_t reduce_affine_ws(int64_t n_rest, int64_t nout) {
  return n_rest <= kWarpRun ? 0 : ws_for(n_rest, nout);
}

int32_t launch_reduce_affine(int32_t dtype, const void *in, const Plan &p, void *out, int32_t flags,
                             void *ws, size_t ws_bytes, desc_stream_t st) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  return with_accumulator(dtype, flags, [&](auto tag) {
    using A = typename decltype(tag)::Acc;
    using T = typename decltype(tag)::Elem;
    return run_affine<A, T>(static_cast<const T *>(in), p, static_cast<T *>(out), ws, ws_bytes, s);
  });
}

int32_t launch_split_reduce_transpose(int32_t dtype, const void *in, int64_t start, int64_t seg_stride,
                                      int64_t len, int64_t nout, void *out, void *ws, size_t ws_bytes,
                                      const float *tin, float *tout, int64_t R, int64_t C, desc_stream_t st) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  if (len <= kWarpRun) return DESC_ERR_UNSUPPORTED;   // the chunked schedule only
  const Cand &cd = kCands[0];
  const int64_t chunks = chunks_for(len, nout, cd);
  uint2 *partials = nullptr;
  unsigned *counters = nullptr;
  if (chunks > 1) {
    if (!ws || ws_bytes < ws_for(len, nout)) return DESC_ERR_WORKSPACE;
    partials = static_cast<uint2 *>(ws);
    counters = reinterpret_cast<unsigned *>(static_cast<char *>(ws) +
                                            align256(size_t(nout) * max_chunks(len, nout) * sizeof(uint2)));
    DESC_CUDA_TRY(cudaMemsetAsync(counters, 0, size_t(nout) * sizeof(unsigned), s));
  }
  const int64_t nred = nout * chunks;
  SplitTranspose tr{tin, tout, R, C, (C + 63) / 64};
  const int64_t ntr = tr.gx * ((R + 63) / 64);
  if (nred + ntr >= (int64_t(1) << 31)) return DESC_ERR_UNSUPPORTED;
  const unsigned grid = (unsigned)(nred + ntr);
  if (grid == 0) return DESC_OK;
  if (dtype == DESC_I32)
    split_reduce_transpose_kernel<AccI32, int32_t><<<grid, kThreads, 0, s>>>(
        static_cast<const int32_t *>(in), start, seg_stride, len, chunks, static_cast<int32_t *>(out), partials,
        counters, nred, tr);
  else
    split_reduce_transpose_kernel<AccF32, float><<<grid, kThreads, 0, s>>>(
        static_cast<const float *>(in), start, seg_stride, len, chunks, static_cast<float *>(out), partials,
        counters, nred, tr);
  DESC_CUDA_TRY(cudaGetLastError());
  return DESC_OK;
}

namespace {
__global__ void fill_u32_kernel(uint32_t *out, int64_t n, uint32_t v) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = v;
}
}  // namespace

int32_t fill_identity(void *out, int64_t count, int32_t dtype, int32_t flags, desc_stream_t st) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  if (count <= 0) return DESC_OK;
  uint32_t v = 0u;                                                          // sum, or, xor
  if (flags & DESC_MAX) v = dtype == DESC_I32 ? 0x80000000u : 0xff800000u;   // INT32_MIN, -inf
  if (flags & DESC_MIN) v = dtype == DESC_I32 ? 0x7fffffffu : 0x7f800000u;   // INT32_MAX, +inf
  if (flags & DESC_PROD) v = dtype == DESC_I32 ? 1u : 0x3f800000u;           // 1, 1.0f
  if (flags & (DESC_AND | DESC_ARGMAX | DESC_ARGMIN)) v = 0xffffffffu;       // all ones; index -1
  if (v == 0u) return cudaMemsetAsync(out, 0, size_t(count) * 4, s) == cudaSuccess ? DESC_OK : DESC_ERR_CUDA;
  const int64_t blocks = std::min<int64_t>((count + 255) / 256, 4096);
  fill_u32_kernel<<<(unsigned)blocks, 256, 0, s>>>(static_cast<uint32_t *>(out), count, v);
  DESC_CUDA_TRY(cudaGetLastError());
  return DESC_OK;
}

}  // namespace desc
