// Inclusive scan kernels: single pass, decoupled look-back.
//
// Each CTA takes the next tile (TILE = THREADS * ITEMS elements) from an
// atomic ticket, so every tile's predecessors are already running or done.
// In the tile: 128-bit loads, a sequential segmented scan of each thread's
// ITEMS, a warp scan with shuffles and a scan of the warp totals in shared
// memory.  The tile then publishes its total and looks back over earlier
// tiles (one warp, 32 tiles per step) until it meets a tile that has
// published its inclusive prefix; it adds what it saw, publishes its own
// inclusive prefix, and applies the carry.
//
// Segments: head flags mark segment starts (none for one segment; every
// `period` elements; or CSR offsets).  A tile that contains a head publishes
// its inclusive value at once (nothing before the head can change it).
//
// Published words (64 bit, single-copy atomic): status in bits 63..62
// (1 = tile total, 2 = inclusive prefix), value bits in 31..0.  FP32 values
// travel as an unevaluated (hi, lo) pair, in two words that both carry the
// status; a reader accepts them only when the two statuses agree.  The carry
// is accumulated with error-free transformations, so the per-element error
// stays within (ITEMS + log2 THREADS + 2) ulp-sized terms of sum |x|.
//
// Every wait is bounded: a waiting warp gives up after a clock64 budget (or
// as soon as another tile has given up), records DESC_ERR_DEVICE_TIMEOUT in
// the device status word, and its CTA leaves without writing.
#include <algorithm>

#include "k_common.cuh"

namespace desc {

__device__ int g_scan_status;

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;
constexpr unsigned long long kStatAgg = 1ull, kStatIncl = 2ull;
constexpr long long kBudgetCycles = 1ll << 31;      // about one second
constexpr long long kDebugBudgetCycles = 1ll << 26; // tens of milliseconds

enum Mode { PLAIN = 0, PERIODIC = 1, CSR = 2 };

struct TileState {
  unsigned long long w0, w1;
};

struct ScanWs {
  unsigned ticket;
  unsigned abort;
};

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Carry value: int32 modulo 2^32, or an FP32 (hi, lo) pair.
template <class T> struct Carry;
template <> struct Carry<int32_t> {
  uint32_t v;
  __device__ static Carry zero() { return {0u}; }
  __device__ static Carry of(int32_t x) { return {(uint32_t)x}; }
  __device__ Carry plus(const Carry &o) const { return {v + o.v}; }
  __device__ Carry shfl_down(int off) const { return {__shfl_down_sync(0xffffffffu, v, off)}; }
  __device__ uint32_t hi_bits() const { return v; }
  __device__ uint32_t lo_bits() const { return 0u; }
  __device__ static Carry from_bits(uint32_t h, uint32_t) { return {h}; }
};
template <> struct Carry<float> {
  float hi, lo;
  __device__ static Carry zero() { return {0.f, 0.f}; }
  __device__ static Carry of(float x) { return {x, 0.f}; }
  __device__ Carry plus(const Carry &o) const {
    float s, e;
    two_sum(hi, o.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, o.lo));
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
  }
  __device__ Carry shfl_down(int off) const {
    return {__shfl_down_sync(0xffffffffu, hi, off), __shfl_down_sync(0xffffffffu, lo, off)};
  }
  __device__ uint32_t hi_bits() const { return __float_as_uint(hi); }
  __device__ uint32_t lo_bits() const { return __float_as_uint(lo); }
  __device__ static Carry from_bits(uint32_t h, uint32_t l) { return {__uint_as_float(h), __uint_as_float(l)}; }
};

template <class T>
__device__ __forceinline__ T add_t(T a, T b);
template <>
__device__ __forceinline__ int32_t add_t(int32_t a, int32_t b) { return (int32_t)((uint32_t)a + (uint32_t)b); }
template <>
__device__ __forceinline__ float add_t(float a, float b) { return __fadd_rn(a, b); }

// x + carry, the carry added last so its low part is not lost.
__device__ __forceinline__ int32_t apply_carry(int32_t x, const Carry<int32_t> &c) {
  return (int32_t)((uint32_t)x + c.v);
}
__device__ __forceinline__ float apply_carry(float x, const Carry<float> &c) {
  return __fadd_rn(c.hi, __fadd_rn(c.lo, x));
}

template <class T>
__device__ __forceinline__ void publish(TileState *st, unsigned long long status, const Carry<T> &c) {
  const unsigned long long tag = status << 62;
  st_relaxed(&st->w0, tag | c.hi_bits());
  if (sizeof(Carry<T>) > 4) st_relaxed(&st->w1, tag | c.lo_bits());
}

template <class T> struct VecOf;
template <> struct VecOf<int32_t> { using type = int4; };
template <> struct VecOf<float> { using type = float4; };

struct ScanArgs {
  int64_t n;
  int64_t period;          // PERIODIC: segment length
  const int64_t *offsets;  // CSR: nseg + 1 offsets
  int64_t nseg;
  void *sums;              // CSR: per-segment totals (may be null)
  int32_t debug;           // 1: tile 1 never publishes (tests the timeout path)
  int32_t vec;             // in and out are 16-byte aligned: 128-bit accesses
};

// Looks back from tile `tile` (warp 0 only).  Returns false on timeout.
template <class T>
__device__ bool look_back(TileState *states, int64_t tile, ScanWs *ws, long long budget,
                          Carry<T> &prefix) {
  const int lane = threadIdx.x & 31;
  Carry<T> acc = Carry<T>::zero();
  int64_t j = tile - 1;   // nearest predecessor not yet folded in
  const long long t0 = clock64();
  while (true) {
    const int64_t me = j - lane;
    unsigned long long w0 = 0, w1 = 0, st = 0;
    while (true) {
      if (me >= 0) {
        w0 = ld_relaxed(&states[me].w0);
        st = w0 >> 62;
        if (sizeof(Carry<T>) > 4 && st != 0) {
          w1 = ld_relaxed(&states[me].w1);
          if ((w1 >> 62) != st) st = 0;   // torn pair: read again
        }
      } else {
        st = kStatIncl;                   // before tile 0: empty prefix
        w0 = 0; w1 = 0;
      }
      if (__all_sync(0xffffffffu, st != 0)) break;
      int give_up = 0;
      if (lane == 0)
        give_up = (*(volatile unsigned *)&ws->abort != 0u) || (clock64() - t0 > budget);
      give_up = __shfl_sync(0xffffffffu, give_up, 0);
      if (give_up) {
        if (lane == 0) {
          atomicExch(&ws->abort, 1u);
          atomicCAS(&g_scan_status, 0, (int)DESC_ERR_DEVICE_TIMEOUT);
        }
        return false;
      }
      __nanosleep(64);
    }
    const unsigned incl = __ballot_sync(0xffffffffu, st == kStatIncl);
    const int stop = incl ? __ffs(incl) - 1 : 31;     // nearest inclusive prefix
    Carry<T> mine = (lane <= stop) ? Carry<T>::from_bits((uint32_t)w0, (uint32_t)w1) : Carry<T>::zero();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mine = mine.plus(mine.shfl_down(off));
    acc = acc.plus(Carry<T>{mine});
    if (incl) break;
    j -= 32;
  }
  prefix = acc;
  return true;
}

template <class T, int MODE>
__global__ void __launch_bounds__(kThreads) scan_kernel(const T *in, T *out,
                                                        ScanArgs args, ScanWs *ws,
                                                        TileState *states) {
  using V = typename VecOf<T>::type;
  __shared__ int64_t sh_tile;
  __shared__ T sh_wval[kThreads / 32];
  __shared__ int sh_wflag[kThreads / 32];
  __shared__ Carry<T> sh_prefix;
  __shared__ int sh_ok;
  __shared__ unsigned sh_heads[kTile / 32];
  __shared__ int64_t sh_seg0;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    sh_tile = atomicAdd(&ws->ticket, 1u);
    sh_ok = 1;
  }
  __syncthreads();
  const int64_t tile = sh_tile;
  const int64_t t0 = tile * kTile;
  const int64_t n = args.n;
  const bool full = t0 + kTile <= n;
  const int64_t g0 = t0 + int64_t(tid) * kItems;

  // ---- head flags of this thread's items (bit i = item i starts a segment)
  unsigned hmask = 0u;
  if (MODE == PERIODIC) {
    int64_t r = g0 % args.period;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      if (r == 0) hmask |= 1u << i;
      if (++r == args.period) r = 0;
    }
  } else if (MODE == CSR) {
    for (int i = tid; i < kTile / 32; i += kThreads) sh_heads[i] = 0u;
    // segment containing t0: largest s with offsets[s] <= t0 (warp 0 search)
    if (warp == 0) {
      int64_t lo = 0, hi = args.nseg;   // answer in [lo, hi)
      while (hi - lo > 1) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t probe = lo + int64_t(lane) * step;
        const bool le = probe < hi && args.offsets[probe] <= t0;
        const unsigned m = __ballot_sync(0xffffffffu, le);
        const int last = 31 - __clz(m);      // lane 0 always qualifies (offsets[lo] <= t0)
        lo = lo + int64_t(last) * step;
        hi = std::min<int64_t>(hi, lo + step);
      }
      if (lane == 0) sh_seg0 = lo;
    }
    __syncthreads();
    // heads: offsets[s] for s > seg0 with offsets[s] < t0 + kTile
    const int64_t tend = std::min<int64_t>(t0 + kTile, n);
    for (int64_t s = sh_seg0 + 1 + tid; s < args.nseg; s += kThreads) {
      const int64_t b = args.offsets[s];
      if (b >= tend) break;
      const int64_t rel = b - t0;
      atomicOr(&sh_heads[rel >> 5], 1u << (rel & 31));
    }
    if (tid == 0 && args.offsets[sh_seg0] == t0) atomicOr(&sh_heads[0], 1u);
    __syncthreads();
    const int64_t rel0 = int64_t(tid) * kItems;
    hmask = (sh_heads[rel0 >> 5] >> (rel0 & 31)) & ((1u << kItems) - 1u);
  }

  // ---- load and scan this thread's items
  T v[kItems];
  if (full && args.vec) {
    const V *p = reinterpret_cast<const V *>(in + g0);
#pragma unroll
    for (int q = 0; q < kItems / 4; ++q) {
      const V x = ld_stream(p + q);
      v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < kItems; ++i) v[i] = (g0 + i < n) ? in[g0 + i] : T(0);
  }
#pragma unroll
  for (int i = 1; i < kItems; ++i)
    if (!((hmask >> i) & 1u)) v[i] = add_t(v[i - 1], v[i]);
  int f = hmask != 0u;
  T a = v[kItems - 1];

  // ---- warp inclusive scan of (flag, value) with the segmented operator
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const T au = __shfl_up_sync(0xffffffffu, a, off);
    const int fu = __shfl_up_sync(0xffffffffu, f, off);
    if (lane >= off) {
      if (!f) a = add_t(au, a);
      f |= fu;
    }
  }
  if (lane == 31) {
    sh_wval[warp] = a;
    sh_wflag[warp] = f;
  }
  // thread-exclusive within the warp
  T ex = __shfl_up_sync(0xffffffffu, a, 1);
  int exf = __shfl_up_sync(0xffffffffu, f, 1);
  if (lane == 0) { ex = T(0); exf = 0; }
  __syncthreads();
  // ---- scan of the warp totals (warp 0), exclusive per warp
  if (warp == 0) {
    T wa = lane < kThreads / 32 ? sh_wval[lane] : T(0);
    int wf = lane < kThreads / 32 ? sh_wflag[lane] : 0;
#pragma unroll
    for (int off = 1; off < kThreads / 32; off <<= 1) {
      const T au = __shfl_up_sync(0xffffffffu, wa, off);
      const int fu = __shfl_up_sync(0xffffffffu, wf, off);
      if (lane >= off) {
        if (!wf) wa = add_t(au, wa);
        wf |= fu;
      }
    }
    T we = __shfl_up_sync(0xffffffffu, wa, 1);
    int wfe = __shfl_up_sync(0xffffffffu, wf, 1);
    if (lane == 0) { we = T(0); wfe = 0; }
    const T tile_val = __shfl_sync(0xffffffffu, wa, kThreads / 32 - 1);
    const int tile_flag = __shfl_sync(0xffffffffu, wf, kThreads / 32 - 1);
    __syncwarp();
    if (lane < kThreads / 32) {
      sh_wval[lane] = we;
      sh_wflag[lane] = wfe;
    }
    // ---- publish, then look back when the tile's first item needs a carry
    TileState *mine = &states[tile];
    const bool stall = args.debug && tile == 1;
    const bool head_first = (hmask & 1u) && tid == 0;   // lane 0 of warp 0 holds item 0
    const bool first_is_head = __shfl_sync(0xffffffffu, head_first ? 1 : 0, 0) != 0;
    Carry<T> prefix = Carry<T>::zero();
    bool ok = true;
    if (tile == 0 || tile_flag) {
      if (lane == 0 && !stall) publish<T>(mine, kStatIncl, Carry<T>::of(tile_val));
      if (tile != 0 && !first_is_head)
        ok = look_back<T>(states, tile, ws, args.debug ? kDebugBudgetCycles : kBudgetCycles, prefix);
    } else {
      if (lane == 0 && !stall) publish<T>(mine, kStatAgg, Carry<T>::of(tile_val));
      ok = look_back<T>(states, tile, ws, args.debug ? kDebugBudgetCycles : kBudgetCycles, prefix);
      if (ok && lane == 0 && !stall) publish<T>(mine, kStatIncl, prefix.plus(Carry<T>::of(tile_val)));
    }
    if (lane == 0) {
      sh_prefix = prefix;
      sh_ok = ok ? 1 : 0;
    }
  }
  __syncthreads();
  if (!sh_ok) return;

  // ---- combine: warp-exclusive, then thread-exclusive, then the tile carry
  const T wex = sh_wval[warp];
  const int wexf = sh_wflag[warp];
  if (warp > 0 && !exf) ex = add_t(wex, ex);       // prefix of this thread within the tile
  if (warp > 0) exf |= wexf;
  const Carry<T> pre = sh_prefix;
  const bool use_ex = (warp > 0) || (lane > 0);
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    // items after this thread's first head are already final
    if ((hmask & ((2u << i) - 1u)) == 0u) {
      T x = use_ex ? add_t(ex, v[i]) : v[i];
      v[i] = exf ? x : apply_carry(x, pre);
    }
  }
  if (full && args.vec) {
    V *p = reinterpret_cast<V *>(out + g0);
#pragma unroll
    for (int q = 0; q < kItems / 4; ++q) {
      V x;
      x.x = v[4 * q]; x.y = v[4 * q + 1]; x.z = v[4 * q + 2]; x.w = v[4 * q + 3];
      __stcs(p + q, x);
    }
  } else {
#pragma unroll
    for (int i = 0; i < kItems; ++i)
      if (g0 + i < n) out[g0 + i] = v[i];
  }

  // ---- CSR: totals of the segments ending in this tile, read back from out
  if (MODE == CSR && args.sums) {
    __syncthreads();
    T *sums = static_cast<T *>(args.sums);
    const int64_t tend = std::min<int64_t>(t0 + kTile, n);
    for (int64_t s = sh_seg0 + tid; s < args.nseg; s += kThreads) {
      const int64_t b = args.offsets[s], e = args.offsets[s + 1];
      if (b >= tend) break;
      if (e > b && e - 1 >= t0 && e - 1 < tend) sums[s] = __ldcg(out + (e - 1));
    }
    // empty segments: this tile's share of the segment index space
    const int64_t ntiles = (n + kTile - 1) / kTile;
    for (int64_t s = tile * kThreads + tid; s < args.nseg; s += ntiles * kThreads)
      if (args.offsets[s + 1] == args.offsets[s]) sums[s] = T(0);
  }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

template <class T, int MODE>
int32_t run_scan(const T *in, T *out, const ScanArgs &a, void *ws, size_t ws_bytes, cudaStream_t s) {
  const int64_t ntiles = (a.n + kTile - 1) / kTile;
  if (ntiles == 0) return DESC_OK;
  const size_t need = align256(sizeof(ScanWs)) + size_t(ntiles) * sizeof(TileState);
  if (!ws || ws_bytes < need) return DESC_ERR_WORKSPACE;
  if (ntiles >= (int64_t(1) << 31)) return DESC_ERR_UNSUPPORTED;
  DESC_CUDA_TRY(cudaMemsetAsync(ws, 0, need, s));
  ScanWs *w = static_cast<ScanWs *>(ws);
  TileState *st = reinterpret_cast<TileState *>(static_cast<char *>(ws) + align256(sizeof(ScanWs)));
  scan_kernel<T, MODE><<<(unsigned)ntiles, kThreads, 0, s>>>(in, out, a, w, st);
  DESC_CUDA_TRY(cudaGetLastError());
  return DESC_OK;
}

}  // namespace

int32_t scan_status_take() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_scan_status, sizeof(int)) != cudaSuccess) return DESC_ERR_CUDA;
  if (v != 0 && cudaMemcpyToSymbol(g_scan_status, &z, sizeof(int)) != cudaSuccess) return DESC_ERR_CUDA;
  return v;
}

size_t scan_contig_ws(int32_t /*dtype*/, int64_t n) {
  const int64_t ntiles = (n + kTile - 1) / kTile;
  return align256(sizeof(ScanWs)) + size_t(ntiles) * sizeof(TileState);
}

int32_t launch_scan_contig(int32_t dtype, const void *in, void *out, int64_t n, int64_t period,
                           int32_t flags, void *ws, size_t ws_bytes, desc_stream_t st) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  ScanArgs a{};
  a.n = n;
  a.period = period;
  a.debug = (flags & DESC_DEBUG_STALL_TILE) ? 1 : 0;
  a.vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
  const bool periodic = period > 0 && period < n;
  if (dtype == DESC_I32) {
    auto i = static_cast<const int32_t *>(in);
    auto o = static_cast<int32_t *>(out);
    return periodic ? run_scan<int32_t, PERIODIC>(i, o, a, ws, ws_bytes, s)
                    : run_scan<int32_t, PLAIN>(i, o, a, ws, ws_bytes, s);
  }
  auto i = static_cast<const float *>(in);
  auto o = static_cast<float *>(out);
  return periodic ? run_scan<float, PERIODIC>(i, o, a, ws, ws_bytes, s)
                  : run_scan<float, PLAIN>(i, o, a, ws, ws_bytes, s);
}

size_t scan_csr_ws(int64_t n) { return scan_contig_ws(DESC_F32, n); }

int32_t launch_scan_csr(int32_t dtype, const void *in, void *out, int64_t n, const int64_t *offsets,
                        int64_t nseg, void *sums, int32_t flags, void *ws, size_t ws_bytes,
                        desc_stream_t st) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  ScanArgs a{};
  a.n = n;
  a.offsets = offsets;
  a.nseg = nseg;
  a.sums = sums;
  a.debug = (flags & DESC_DEBUG_STALL_TILE) ? 1 : 0;
  a.vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
  if (dtype == DESC_I32)
    return run_scan<int32_t, CSR>(static_cast<const int32_t *>(in), static_cast<int32_t *>(out), a,
                                  ws, ws_bytes, s);
  return run_scan<float, CSR>(static_cast<const float *>(in), static_cast<float *>(out), a, ws,
                              ws_bytes, s);
}

}  // namespace desc
