// Scan kernels of libdesc and their host-side launch templates, shared by
// the translation units that instantiate them: k_scan.cu (sums, maxima and
// minima over contiguous runs and CSR segments), k_scan_ops.cu (products and
// bitwise operators), k_scan_mapped.cu (those scans through a lowered map)
// and k_scan_map.cu (the one-tile map scan, the arg operators and the
// per-segment groups).  Everything here has internal linkage: each unit has
// its own device status word and reports it through take_status_word().
//
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
// Published words (64 bit, single-copy atomic, so one load reads a whole
// state): status in bits 63..62 (1 = tile total, 2 = inclusive prefix) and
// the value.  FP32 carries travel as an unevaluated (hi, lo) pair and are
// accumulated with error-free transformations, so the per-element error
// stays within (ITEMS + log2 THREADS + 2) ulp-sized terms of sum |x|.
//
// Every wait is bounded: a waiting warp gives up after a clock64 budget (or
// as soon as another tile has given up), records DESC_ERR_DEVICE_TIMEOUT in
// the device status word, and its CTA leaves without writing.
#pragma once

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "k_common.cuh"

namespace desc {
namespace {

// This translation unit's device status word (DESC_ERR_DEVICE_TIMEOUT).
__device__ int g_scan_status;

constexpr unsigned long long kStatAgg = 1ull, kStatIncl = 2ull;
constexpr long long kBudgetCycles = 1ll << 31;      // about one second
constexpr long long kDebugBudgetCycles = 1ll << 26; // tens of milliseconds
constexpr unsigned kGoSpins = 1u << 16;                // x 64 ns: the look-back start wait

enum Mode { PLAIN = 0, PERIODIC = 1, CSR = 2 };

struct alignas(kScanTileStateBytes) TileState {
  unsigned long long w;
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

// One 64-bit word per tile: status in bits 63..62, value below.  int32:
// the value in bits 31..0.  FP32: hi in bits 31..0 and lo, with its two
// lowest mantissa bits dropped (a relative change below 2^-21 of a term that
// is itself below half an ulp of hi), in bits 61..32.
__device__ __forceinline__ unsigned long long pack(unsigned long long status, const Carry<int32_t> &c) {
  return (status << 62) | c.v;
}
__device__ __forceinline__ unsigned long long pack(unsigned long long status, const Carry<float> &c) {
  return (status << 62) | ((unsigned long long)(__float_as_uint(c.lo) >> 2) << 32) | __float_as_uint(c.hi);
}
template <class T>
__device__ __forceinline__ Carry<T> unpack(unsigned long long w);
template <>
__device__ __forceinline__ Carry<int32_t> unpack(unsigned long long w) { return {(uint32_t)w}; }
template <>
__device__ __forceinline__ Carry<float> unpack(unsigned long long w) {
  return {__uint_as_float((uint32_t)w), __uint_as_float((uint32_t)((w >> 32) & 0x3FFFFFFFull) << 2)};
}

// Scan operators.  O::C is the carry type a look-back folds; apply(x, c)
// combines a carry with an element's in-tile prefix; pack/unpack place a
// carry in the 62 value bits of a tile state.
template <class T>
struct SumOp {                          // sum: int32 modulo 2^32, FP32 with compensated carries
  using C = Carry<T>;
  __device__ static T id() { return T(0); }
  __device__ static T comb(T a, T b) { return add_t(a, b); }
  __device__ static T apply(T x, const C &c) { return apply_carry(x, c); }
  __device__ static unsigned long long pack(unsigned long long st, const C &c) { return desc::pack(st, c); }
  __device__ static C unpack(unsigned long long w) { return desc::unpack<T>(w); }
};

// Value operators other than the sum: maximum, minimum (FP32 ignores NaN
// operands, IEEE maxNum / minNum), product (int32 modulo 2^32, FP32 in FP32),
// bitwise and / or / xor (int32).  Carries are plain values.
enum ValKind { kMaxOp = 0, kMinOp = 1, kProdOp = 2, kAndOp = 3, kOrOp = 4, kXorOp = 5 };
template <class T, int K>
struct ValOp {
  __device__ static T id() {
    if constexpr (std::is_same<T, float>::value) {
      if (K == kMaxOp) return -__int_as_float(0x7f800000);
      if (K == kMinOp) return __int_as_float(0x7f800000);
      return 1.0f;                                      // product
    } else {
      if (K == kMaxOp) return INT32_MIN;
      if (K == kMinOp) return INT32_MAX;
      if (K == kProdOp) return 1;
      if (K == kAndOp) return -1;
      return 0;                                         // or, xor
    }
  }
  __device__ static T comb(T a, T b) {
    if constexpr (std::is_same<T, float>::value) {
      if (K == kMaxOp) return fmaxf(a, b);
      if (K == kMinOp) return fminf(a, b);
      return __fmul_rn(a, b);
    } else {
      const uint32_t x = (uint32_t)a, y = (uint32_t)b;
      if (K == kMaxOp) return max(a, b);
      if (K == kMinOp) return min(a, b);
      if (K == kProdOp) return (int32_t)(x * y);
      if (K == kAndOp) return (int32_t)(x & y);
      if (K == kOrOp) return (int32_t)(x | y);
      return (int32_t)(x ^ y);
    }
  }
  struct C {
    T v;
    __device__ static C zero() { return {ValOp::id()}; }
    __device__ static C of(T x) { return {x}; }
    __device__ C plus(const C &o) const { return {ValOp::comb(v, o.v)}; }   // commutative operators
    __device__ C shfl_down(int off) const { return {__shfl_down_sync(0xffffffffu, v, off)}; }
  };
  __device__ static T apply(T x, const C &c) { return comb(c.v, x); }
  __device__ static unsigned long long pack(unsigned long long st, const C &c) {
    return (st << 62) | (unsigned long long)__builtin_bit_cast(uint32_t, c.v);
  }
  __device__ static C unpack(unsigned long long w) { return {__builtin_bit_cast(T, (uint32_t)w)}; }
};
template <class T, bool MAX>
using ExtOp = ValOp<T, MAX ? kMaxOp : kMinOp>;

template <class O>
__device__ __forceinline__ void publish(TileState *st, unsigned long long status, const typename O::C &c) {
  st_relaxed(&st->w, O::pack(status, c));
}

// A lowered map for the scans that read and write through it: point g
// (row-major over the canonical dims) is element map_elem(m, g).
struct MapArgs {
  int32_t nd;                       // dims of the canonical map; 0: element = off + g
  int32_t fast;                     // fewer than 2^32 points: 32-bit decoding
  int64_t off;
  int64_t ext[DESC_MAX_DIMS];
  int64_t st[DESC_MAX_DIMS];
  FastDiv div[DESC_MAX_DIMS];
};

// Maps of two or more dims: decoded dim by dim (out of line: the kernel
// inlines only the one-dim case).
__device__ __noinline__ int64_t map_elem_dims(const MapArgs &m, int64_t g) {
  int64_t e = m.off;
  if (m.fast) {
    uint32_t t = (uint32_t)g;
    for (int d = m.nd - 1; d > 0; --d) {
      const uint32_t q = fast_div(t, m.div[d]);
      e += int64_t(t - q * m.div[d].d) * m.st[d];
      t = q;
    }
    return e + int64_t(t) * m.st[0];
  }
  int64_t t = g;
  for (int d = m.nd - 1; d >= 0; --d) {
    e += (t % m.ext[d]) * m.st[d];
    t /= m.ext[d];
  }
  return e;
}
__device__ __forceinline__ int64_t map_elem(const MapArgs &m, int64_t g) {
  if (m.nd <= 1) return m.off + (m.nd ? g * m.st[0] : g);
  return map_elem_dims(m, g);
}

// Global addressing of the look-back scan: the identity (contiguous runs)
// or a lowered map.
struct RunAddr {
  const MapArgs &m;                                     // not used
  static constexpr bool kAffine = true;                 // addr(g + k) = addr(g) + step(k)
  __device__ int64_t operator()(int64_t g) const { return g; }
  __device__ int64_t step(int64_t k) const { return k; }
};
// The look-back scan takes maps of one or two dims, the count fixed at
// compile time (a run-time test of it cost 7 % of the scan), decoded inline
// (launch_scan_mapped checks the ranges):
//   ND = 1: off + g * st[0], as one 32 x 32 -> 64-bit product (g < 2^31,
//           |st[0]| < 2^31);
//   ND = 2: g split by the inner extent with a 32-bit multiply-high division
//           (fewer than 2^32 points).
template <int ND>
struct MapAddr {
  const MapArgs &m;
  static constexpr bool kAffine = ND == 1;              // addr(g + k) = addr(g) + step(k)
  __device__ int64_t step(int64_t k) const { return k * m.st[0]; }
  __device__ int64_t operator()(int64_t g) const {
    if constexpr (ND == 1) {
      return m.off + int64_t(int32_t(g)) * int64_t(int32_t(m.st[0]));
    } else {
      const uint32_t t = (uint32_t)g, q = fast_div(t, m.div[1]);
      return m.off + int64_t(q) * m.st[0] + int64_t(t - q * m.div[1].d) * m.st[1];
    }
  }
};

struct ScanArgs {
  int64_t n;
  int64_t period;          // PERIODIC: segment length
  const int64_t *offsets;  // CSR: nseg + 1 offsets
  int64_t nseg;
  void *sums;              // CSR: per-segment totals (may be null)
  int32_t debug;           // 1: tile 1 never publishes (tests the timeout path)
  int32_t vec;             // 128-bit accesses: 1 ascending, 2 descending chunks (load_sub); 0 none
  FastDiv pdiv;            // PERIODIC: the period, where it is below 2^30 (set by with_period)
};

// The launch arguments with the period's divisor filled in.
inline ScanArgs with_period(ScanArgs a) {
  if (a.period > 0 && a.period < (int64_t(1) << 30)) a.pdiv = make_fastdiv(uint32_t(a.period));
  return a;
}

// PERIODIC: the position in its segment of the point `off` (0 <= off < TILE)
// past a tile start whose own position is r0 (0 <= r0 < period): one
// conditional subtraction where segments are at least a tile long, else a
// 32-bit multiply-high division (the operand is below period + TILE).
template <int TILE>
__device__ __forceinline__ int64_t seg_pos(int64_t r0, int off, const ScanArgs &a) {
  if (a.period >= TILE) {
    const int64_t x = r0 + off;
    return x >= a.period ? x - a.period : x;
  }
  const uint32_t x = uint32_t(r0) + uint32_t(off);
  return int64_t(x - fast_div(x, a.pdiv) * a.pdiv.d);
}

// Bit i (i < COUNT) set where point i of a run starting at position pos
// (0 <= pos < period) of its segment is a segment head.
template <int COUNT>
__device__ __forceinline__ unsigned seg_heads(int64_t pos, int64_t period) {
  unsigned hm = 0u;
  for (int64_t i = pos == 0 ? 0 : period - pos; i < COUNT; i += period) hm |= 1u << i;
  return hm;
}

// Looks back from tile `tile` (one warp).  Each poll reads a window of
// 32 x kSlots tile states (lane l takes kSlots consecutive ones); everything
// up to the nearest inclusive prefix in the window must have published
// before the window is folded in.  Failed polls back off exponentially, which
// keeps the hot tile states from being flooded.  Returns false on timeout.
constexpr int kSlots = 1;

template <class O>
__device__ bool look_back(TileState *states, int64_t tile, ScanWs *ws, long long budget,
                          typename O::C &prefix) {
  using CT = typename O::C;
  const int lane = threadIdx.x & 31;
  CT acc = CT::zero();
  int64_t j = tile - 1;   // nearest predecessor not yet folded in
  const long long t0 = clock64();
  unsigned polls = 0;
  while (true) {
    unsigned long long w[kSlots];
    int stop;
    unsigned incl_lanes;
    while (true) {
#pragma unroll
      for (int k = 0; k < kSlots; ++k) {
        const int64_t me = j - (lane * kSlots + k);
        w[k] = me >= 0 ? ld_relaxed(&states[me].w) : (kStatIncl << 62);   // before tile 0: empty
      }
      int kin = kSlots;                                 // nearest inclusive slot of this lane
#pragma unroll
      for (int k = kSlots - 1; k >= 0; --k)
        if ((w[k] >> 62) == kStatIncl) kin = k;
      incl_lanes = __ballot_sync(0xffffffffu, kin < kSlots);
      const int first = incl_lanes ? __ffs(incl_lanes) - 1 : 31;
      const int kfirst = __shfl_sync(0xffffffffu, kin, first);
      stop = incl_lanes ? first * kSlots + kfirst : 32 * kSlots - 1;
      bool ready = true;
#pragma unroll
      for (int k = 0; k < kSlots; ++k)
        if (lane * kSlots + k <= stop && (w[k] >> 62) == 0) ready = false;
      if (__all_sync(0xffffffffu, ready)) break;
      int give_up = 0;
      ++polls;
      if (lane == 0 && (polls & 31) == 0)      // the abort flag is one more L2 round trip
        give_up = (*(volatile unsigned *)&ws->abort != 0u) || (clock64() - t0 > budget);
      give_up = __shfl_sync(0xffffffffu, give_up, 0);
      if (give_up) {
        if (lane == 0) {
          atomicExch(&ws->abort, 1u);
          atomicCAS(&g_scan_status, 0, (int)DESC_ERR_DEVICE_TIMEOUT);
        }
        return false;
      }
      __nanosleep(min(32u << min(polls, 5u), 1024u));   // exponential back-off
    }
    CT mine = CT::zero();
#pragma unroll
    for (int k = 0; k < kSlots; ++k)
      if (lane * kSlots + k <= stop) mine = mine.plus(O::unpack(w[k]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mine = mine.plus(mine.shfl_down(off));
    acc = acc.plus(mine);
    if (incl_lanes) break;
    j -= 32 * kSlots;
  }
  prefix = acc;
  return true;
}

// ---- asynchronous tile copies (cp.async) into swizzled shared memory ----
// A sub-tile is 1024 chunks of 16 bytes.  Chunk j sits in slot
// j ^ ((j >> 3) & 3): within each 128-byte row the slots are permuted so
// that both the striped accesses (lane l on chunk base + l, used to move
// data to and from global memory with full 128-byte lines) and the blocked
// accesses (thread t on chunks 4t..4t+3, used by the scan) hit 8 distinct
// 16-byte bank groups in every phase of 8 lanes, without padding.
__device__ __forceinline__ int chunk_off(int j) { return 16 * (j ^ ((j >> 3) & 3)); }

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// A CTA scans one tile of kSub * SUB elements: SUB sub-tiles of kSub
// elements (kThreads threads x kItems items), each staged in shared memory.
// Large tiles matter: decoupled look-back serves at most about one window of
// tiles per L2 round trip, so the bytes per tile set the attainable rate.
constexpr int kThreads = 256;                       // scanning threads
constexpr int kItems = 16;                          // elements per thread and sub-tile
constexpr int kWarps = kThreads / 32;
constexpr int kSub = kThreads * kItems;             // elements per sub-tile
constexpr int kSubChunks = kSub / 4;                // 16-byte chunks per sub-tile
constexpr int kStageBytes = 16 * kSubChunks;

__device__ __forceinline__ void compute_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory"); }
// CSR: the compute warps and the look-back warp, once the tile's segment heads are marked.
__device__ __forceinline__ void heads_bar() { asm volatile("bar.sync 2, %0;" ::"n"(kThreads + 32) : "memory"); }

// Start copying kSub elements from g_start (elements past n read as zero);
// point g is in[addr(g)].  vec: 0, one element a copy; 1, four consecutive
// points are four ascending elements on a 16-byte boundary; 2, four
// descending ones (a reversed run), copied whole and so stored in the chunk
// last point first -- every chunk of such a stage is in that order, the
// partial one at the end too, and readers swap it (DESC: the caller may pass 2).
template <class T, bool DESC = false, class A>
__device__ __forceinline__ void load_sub(unsigned char *stage, const T *in, int64_t g_start,
                                         int64_t n, int vec, const A &addr) {
  // an affine map: chunk q's element from the first chunk's by q steps
  const int64_t e0 = A::kAffine ? addr(g_start + 4 * int64_t(threadIdx.x)) : 0;
  const int64_t de = A::kAffine ? addr.step(4 * kThreads) : 0;
#pragma unroll
  for (int q = 0; q < kSubChunks / kThreads; ++q) {
    const int j = q * kThreads + threadIdx.x;
    const int64_t g = g_start + 4 * int64_t(j);
    const int64_t eg = A::kAffine ? e0 + q * de : addr(g);   // the element of point g
    unsigned char *dst = stage + chunk_off(j);
    if (vec == 1) {
      const int64_t rem = n - g;
      const int bytes = rem >= 4 ? 16 : (rem > 0 ? int(rem) * 4 : 0);
      cp_async16(dst, bytes ? static_cast<const void *>(in + eg) : static_cast<const void *>(in), bytes);
    } else if (DESC && vec == 2 && g + 4 <= n) {
      cp_async16(dst, in + (A::kAffine ? eg + addr.step(3) : addr(g + 3)), 16);
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        unsigned char *slot = dst + 4 * (DESC && vec == 2 ? 3 - c : c);
        if (g + c < n) cp_async4(slot, in + (A::kAffine ? eg + addr.step(c) : addr(g + c)));
        else *reinterpret_cast<T *>(slot) = T(0);
      }
    }
  }
}

// A chunk of a stage in point order (see load_sub); only a scan through a
// one-dim map (DESC = true) can have descending chunks.
template <bool DESC>
__device__ __forceinline__ int4 chunk_in_order(int4 x, int vec) {
  if constexpr (DESC) return vec == 2 ? make_int4(x.w, x.z, x.y, x.x) : x;
  return x;
}

__device__ __forceinline__ void cp_async_wait_dyn(int pending) {
  switch (pending) {
    case 0: cp_async_wait<0>(); break;
    case 1: cp_async_wait<1>(); break;
    case 2: cp_async_wait<2>(); break;
    default: cp_async_wait<3>(); break;
  }
}

// The segment containing element t0: the largest s with offsets[s] <= t0
// (one warp, 32-way search).
__device__ __forceinline__ int64_t find_segment(const int64_t *offsets, int64_t nseg, int64_t t0) {
  const int lane = threadIdx.x & 31;
  int64_t lo = 0, hi = nseg;
  while (hi - lo > 1) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t probe = lo + int64_t(lane) * step;
    const bool le = probe < hi && offsets[probe] <= t0;
    const unsigned m = __ballot_sync(0xffffffffu, le);
    const int last = 31 - __clz(m);   // lane 0 always qualifies
    lo = lo + int64_t(last) * step;
    hi = std::min<int64_t>(hi, lo + step);
  }
  return lo;
}

// One CTA per tile, tiles in ticket order.  Warps 0..7 load the tile (one
// cp.async group per sub-tile into padded shared memory, full 128-byte
// lines), scan the sub-tiles in order with an in-tile carry, and publish the
// tile total as soon as it is known.  Warp 8 looks back meanwhile (the prefix
// of a tile does not depend on its data) and publishes the inclusive prefix
// once it has both.  The carry is added during the coalesced store pass, to
// the elements that have no segment start before them in the tile.
// MAPPED (the map's dims, 1 or 2; 0: a contiguous run): points are addressed
// through the lowered map m (in and out are then the base arrays; vec means
// four consecutive points from a multiple of 4 are four consecutive elements
// on a 16-byte boundary).
template <class T, class O, int MODE, int SUB, bool EXCL, int MAPPED>
__global__ void __launch_bounds__(kThreads + 32, 3) scan_kernel(const T *in, T *out, ScanArgs args,
                                                             ScanWs *ws, TileState *states,
                                                             const __grid_constant__ MapArgs m) {
  using CT = typename O::C;
  constexpr int kTile = kSub * SUB;
  extern __shared__ __align__(128) unsigned char ring[];   // SUB stages
  __shared__ int64_t sh_tile;
  __shared__ T sh_wval[kWarps];
  __shared__ int sh_wflag[kWarps];
  __shared__ T sh_carry;                // the tile aggregate, once its sub-tiles are scanned
  __shared__ int sh_carry_flag;
  __shared__ CT sh_prefix;
  __shared__ int sh_ok;
  __shared__ unsigned sh_heads[MODE == CSR ? kTile / 32 : 1];
  __shared__ unsigned short sh_need[MODE == PLAIN ? 1 : SUB * kThreads];  // carry-needed bits
  __shared__ int64_t sh_seg0;
  __shared__ int64_t sh_r0;             // PERIODIC: t0's position in its segment
  __shared__ int sh_tile_heads;         // PERIODIC / CSR: a segment may start in this tile
  __shared__ int sh_any_end;            // CSR: a non-empty segment ends in this tile
  __shared__ int sh_dense;              // CSR: more boundaries than one warp-wide read covers
  __shared__ volatile int sh_go;        // look-back may start polling

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n = args.n;
  const int vec = MAPPED == 1 ? args.vec : (args.vec != 0 ? 1 : 0);   // 2 only through one-dim maps
  using Addr = typename std::conditional<MAPPED == 0, RunAddr, MapAddr<MAPPED == 2 ? 2 : 1>>::type;
  const Addr addr{m};
  if (tid == 0) {
    sh_tile = atomicAdd(&ws->ticket, 1u);
    sh_go = 0;
  }
  if (warp < kWarps) {
    // While the ticket travels: pull into L2 the tile this CTA's index
    // suggests (CTAs take tickets in about the order they start, so a wrong
    // guess is a tile a neighbour loads soon; nothing reads it from here).
    // One prefetch per 32 points: a 128-byte line where the points are
    // contiguous.
    const int64_t guess = int64_t(blockIdx.x) * kTile;
#pragma unroll
    for (int k = 0; k < kTile / 32 / kThreads; ++k) {
      const int64_t g = guess + 32 * int64_t(k * kThreads + tid);
      if (g < n) asm volatile("prefetch.global.L2 [%0];" ::"l"(in + addr(g)));
    }
  }
  __syncthreads();
  const int64_t tile = sh_tile;
  const int64_t t0 = tile * kTile;
  const bool stall = args.debug && tile == 1;

  if (warp == kWarps) {
    // ---- look-back warp: prefix of everything before t0
    bool first_is_head = tile == 0;
    if (MODE == PERIODIC) first_is_head = first_is_head || (t0 % args.period == 0);
    if (MODE == CSR) {
      // The tile's segment heads, found while the compute warps' loads are in
      // flight: zero the bitmap, find the segment holding t0, and mark the
      // boundaries b = offsets[s] in (t0, tend] -- a segment starts at b
      // (b < tend) and segment s - 1 ends at b - 1 -- from one warp-wide read
      // of the next 32 offsets.  Where all 32 lie in the tile there may be
      // more: the compute warps then mark them together (sh_dense).
      for (int i = lane; i < kTile / 32; i += 32) sh_heads[i] = 0u;
      const int64_t tend = std::min<int64_t>(t0 + kTile, n);
      T *sums = static_cast<T *>(args.sums);
      const int64_t s0 = find_segment(args.offsets, args.nseg, t0);
      const int64_t sl = s0 + 1 + lane;
      const int64_t b = sl <= args.nseg ? args.offsets[sl] : INT64_MAX;
      const int64_t bprev = sl <= args.nseg ? args.offsets[sl - 1] : 0;   // lane 0: offsets[s0]
      const bool h0 = __shfl_sync(0xffffffffu, bprev, 0) == t0;           // a segment starts at t0
      const bool dense = __all_sync(0xffffffffu, b <= tend);
      __syncwarp();                                     // bitmap zeroed before marking
      int ends = 0;
      if (!dense && b > t0 && b <= tend) {
        const int64_t rel = b - t0;
        if (b < tend) atomicOr(&sh_heads[rel >> 5], 1u << (rel & 31));
        if (sums) {                                     // empty segments get their total here
          if (bprev == b) sums[sl - 1] = O::id();
          else ends = 1;
        }
      }
      ends = __any_sync(0xffffffffu, ends);
      const bool any_head = __any_sync(0xffffffffu, b > t0 && b < tend);
      if (sums && tile == 0)                            // empty segments before the first element
        for (int64_t q = lane; q < s0; q += 32) sums[q] = O::id();
      if (lane == 0) {
        if (h0) atomicOr(&sh_heads[0], 1u);
        sh_seg0 = s0;
        sh_dense = dense ? 1 : 0;
        sh_any_end = ends;
        sh_tile_heads = (h0 || dense || any_head) ? 1 : 0;
      }
      first_is_head = first_is_head || h0;
      heads_bar();
    }
    CT prefix = CT::zero();
    bool ok = true;
    if (!first_is_head) {
      // Polls made before the predecessors, which started just before this
      // tile, can have published only fail and load the tile states; start
      // once part of this tile's own input has landed (bounded wait).
      for (unsigned i = 0; i < kGoSpins && !sh_go; ++i) __nanosleep(64);
      ok = look_back<O>(states, tile, ws, args.debug ? kDebugBudgetCycles : kBudgetCycles, prefix);
    }
    if (lane == 0) {
      sh_prefix = prefix;
      sh_ok = ok ? 1 : 0;
    }
    __syncthreads();                                    // (S) tile total known
    if (ok && lane == 0 && !stall && tile != 0 && !sh_carry_flag)
      publish<O>(&states[tile], kStatIncl, prefix.plus(CT::of(sh_carry)));
    return;
  }

  // ---- compute warps
#pragma unroll
  for (int s = 0; s < SUB; ++s) {
    load_sub<T, MAPPED == 1>(ring + s * kStageBytes, in, t0 + int64_t(s) * kSub, n, vec, addr);
    cp_async_commit();
  }
  if (tid == 0) {
    sh_carry = O::id();
    sh_carry_flag = 0;
    if (MODE == PERIODIC) {
      sh_r0 = t0 % args.period;                       // one 64-bit division a tile
      sh_tile_heads = sh_r0 == 0 || args.period - sh_r0 < kTile;
    }
  }

  bool tile_heads = false;
  T run_cv = O::id();                                   // the in-tile carry, the same in every thread
  int run_cf = 0;
#pragma unroll 1
  for (int s = 0; s < SUB; ++s) {
    unsigned char *st = ring + s * kStageBytes;
    cp_async_wait_dyn(SUB - 1 - s);                     // sub-tile s has landed (this thread)
    if (MODE == CSR && s == 0) {                        // ... for every thread, and the heads are marked
      heads_bar();
      if (sh_dense) {                                   // many boundaries: all compute threads mark them
        const int64_t tend = std::min<int64_t>(t0 + kTile, n);
        T *sums = static_cast<T *>(args.sums);
        for (int64_t q = sh_seg0 + 1 + tid; q <= args.nseg; q += kThreads) {
          const int64_t b = args.offsets[q];
          if (b > tend) break;
          if (b <= t0) continue;                        // only if the offsets were not sorted
          const int64_t rel = b - t0;
          if (b < tend) atomicOr(&sh_heads[rel >> 5], 1u << (rel & 31));
          if (sums) {
            if (args.offsets[q - 1] == b) sums[q - 1] = O::id();
            else sh_any_end = 1;
          }
        }
        compute_bar();
      }
    } else {
      compute_bar();                                    // ... for every thread; carry visible
    }
    if (s == SUB / 2 && tid == 0) sh_go = 1;
    if (s == 0) tile_heads = MODE != PLAIN && sh_tile_heads;
    // HEADS: the tile may hold segment heads; without them the sub-tile is
    // scanned as a plain run (no flags in the warp and block scans)
    auto sub_tile = [&](auto heads) {
    constexpr bool HEADS = decltype(heads)::value;
    const T cv = run_cv;                                // the in-tile carry before this sub-tile
    const int cf = run_cf;
    unsigned hmask = 0u;
    if constexpr (HEADS) {
      if (MODE == PERIODIC) {
        hmask = seg_heads<kItems>(seg_pos<kTile>(sh_r0, s * kSub + tid * kItems, args), args.period);
      } else if (MODE == CSR) {
        const int rel0 = s * kSub + tid * kItems;
        hmask = (sh_heads[rel0 >> 5] >> (rel0 & 31)) & 0xffffu;
      }
    }
    T v[kItems];
#pragma unroll
    for (int q = 0; q < kItems / 4; ++q) {
      const int4 x = chunk_in_order<MAPPED == 1>(*reinterpret_cast<const int4 *>(st + chunk_off((kItems / 4) * tid + q)), vec);
      v[4 * q] = __builtin_bit_cast(T, x.x);
      v[4 * q + 1] = __builtin_bit_cast(T, x.y);
      v[4 * q + 2] = __builtin_bit_cast(T, x.z);
      v[4 * q + 3] = __builtin_bit_cast(T, x.w);
    }
    if (MODE == PLAIN || hmask == 0u) {                 // no head among the thread's points
#pragma unroll
      for (int i = 1; i < kItems; ++i) v[i] = O::comb(v[i - 1], v[i]);
    } else {
#pragma unroll
      for (int i = 1; i < kItems; ++i)
        if (!((hmask >> i) & 1u)) v[i] = O::comb(v[i - 1], v[i]);
    }
    int f = hmask != 0u;
    T a = v[kItems - 1];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {           // warp scan, segmented operator
      const T au = __shfl_up_sync(0xffffffffu, a, off);
      const int fu = __shfl_up_sync(0xffffffffu, f, off);
      if (lane >= off) {
        if (!f) a = O::comb(au, a);
        f |= fu;
      }
    }
    if (lane == 31) {
      sh_wval[warp] = a;
      if (HEADS) sh_wflag[warp] = f;
    }
    T ex = __shfl_up_sync(0xffffffffu, a, 1);
    int exf = __shfl_up_sync(0xffffffffu, f, 1);
    if (lane == 0) { ex = O::id(); exf = 0; }
    compute_bar();                                      // the sub-tile's warp totals are visible
    // every warp scans the warp totals itself (no warp waits for another, no
    // second barrier); the carry for the next sub-tile stays in registers
    T wa = lane < kWarps ? sh_wval[lane] : O::id();
    int wf = HEADS && lane < kWarps ? sh_wflag[lane] : 0;
#pragma unroll
    for (int off = 1; off < kWarps; off <<= 1) {
      const T au = __shfl_up_sync(0xffffffffu, wa, off);
      const int fu = __shfl_up_sync(0xffffffffu, wf, off);
      if (lane >= off) {
        if (!wf) wa = O::comb(au, wa);
        wf |= fu;
      }
    }
    T we = __shfl_up_sync(0xffffffffu, wa, 1);
    int wfe = __shfl_up_sync(0xffffffffu, wf, 1);
    if (lane == 0) { we = O::id(); wfe = 0; }
    const T sub_val = __shfl_sync(0xffffffffu, wa, kWarps - 1);
    const int sub_flag = __shfl_sync(0xffffffffu, wf, kWarps - 1);
    run_cv = sub_flag ? sub_val : O::comb(cv, sub_val);
    run_cf = cf | sub_flag;
    // prefix of this thread within the tile: carry, then warp, then thread
    const T pv = __shfl_sync(0xffffffffu, we, warp);
    const int pf = __shfl_sync(0xffffffffu, wfe, warp);
    if (!exf) ex = O::comb(pv, ex);
    exf |= pf;                                          // (pf, pv) (+) (exf, ex)
    const T in_tile = exf ? ex : O::comb(cv, ex);
    const int in_flag = exf | cf;
    unsigned need = 0u;                                 // elements with no head before them
    if (MODE == PLAIN || hmask == 0u) {
#pragma unroll
      for (int i = 0; i < kItems; ++i) v[i] = O::comb(in_tile, v[i]);
      need = in_flag ? 0u : 0xffffu;
    } else {
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        if ((hmask & ((2u << i) - 1u)) == 0u) {         // before this thread's first head
          v[i] = O::comb(in_tile, v[i]);
          if (!in_flag) need |= 1u << i;
        }
      }
    }
    if (MODE != PLAIN) sh_need[s * kThreads + tid] = (unsigned short)need;
#pragma unroll
    for (int q = 0; q < kItems / 4; ++q) {
      int4 x;
      x.x = __builtin_bit_cast(int, v[4 * q]);
      x.y = __builtin_bit_cast(int, v[4 * q + 1]);
      x.z = __builtin_bit_cast(int, v[4 * q + 2]);
      x.w = __builtin_bit_cast(int, v[4 * q + 3]);
      *reinterpret_cast<int4 *>(st + chunk_off((kItems / 4) * tid + q)) = x;
    }
    };
    if (tile_heads) sub_tile(std::true_type{});
    else sub_tile(std::false_type{});
  }
  if (tid == 0) {                                       // the tile's aggregate, for the publish and the look-back warp
    sh_carry = run_cv;
    sh_carry_flag = run_cf;
  }
  compute_bar();
  if (tid == 0 && !stall) {
    // publish at once: the inclusive value when nothing before can change it
    // (tile 0, or a tile holding a segment start), else the tile total
    publish<O>(&states[tile], (tile == 0 || sh_carry_flag) ? kStatIncl : kStatAgg, CT::of(sh_carry));
  }
  __syncthreads();                                      // (S) with the look-back warp
  if (!sh_ok) return;                                   // a wait gave up: write nothing

  // ---- coalesced stores, adding the tile carry where needed (the exclusive
  // form, chosen once per launch, shifts each segment by one); a tile with
  // no segment head takes the carry on every element
  const CT pre = sh_prefix;
  const bool no_heads = MODE == PLAIN || !sh_carry_flag;
  const int64_t de = Addr::kAffine ? addr.step(4 * kThreads) : 0;   // elements from chunk j to j + kThreads
#pragma unroll 1
  for (int s = 0; s < SUB; ++s) {
    const unsigned char *st = ring + s * kStageBytes;
    const int64_t e0 = Addr::kAffine ? addr(t0 + int64_t(s) * kSub + 4 * int64_t(tid)) : 0;
#pragma unroll
    for (int q = 0; q < kSubChunks / kThreads; ++q) {
      const int j = q * kThreads + tid;
      const int64_t g = t0 + int64_t(s) * kSub + 4 * int64_t(j);
      const int64_t eg = Addr::kAffine ? e0 + q * de : addr(g);   // the element of point g
      int4 x = *reinterpret_cast<const int4 *>(st + chunk_off(j));
      const unsigned nb = no_heads ? 0xfu : (unsigned(sh_need[s * kThreads + (j >> 2)]) >> ((j & 3) * 4)) & 0xfu;
      T y[4] = {__builtin_bit_cast(T, x.x), __builtin_bit_cast(T, x.y), __builtin_bit_cast(T, x.z),
                __builtin_bit_cast(T, x.w)};
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if ((nb >> c) & 1u) y[c] = O::apply(y[c], pre);
      if (EXCL) {                                       // shift by one within each segment
        const int rel0 = s * kSub + 4 * j;
        T prev = __shfl_up_sync(0xffffffffu, y[3], 1);  // lane - 1 holds chunk j - 1
        if (lane == 0) {
          if (rel0 == 0) {
            prev = O::apply(O::id(), pre);              // everything before the tile
          } else {                                      // from the staged tile
            const int r = rel0 - 1, sb = r / kSub, r2 = r % kSub;
            const T v = reinterpret_cast<const T *>(ring + sb * kStageBytes + chunk_off(r2 / 4))[r2 % 4];
            const bool nd = no_heads || ((sh_need[sb * kThreads + r2 / kItems] >> (r2 % kItems)) & 1u);
            prev = nd ? O::apply(v, pre) : v;
          }
        }
        T e[4];
        const unsigned ph = MODE == PERIODIC ? seg_heads<4>(seg_pos<kTile>(sh_r0, rel0, args), args.period) : 0u;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          bool head;
          if (MODE == PLAIN) head = g + c == 0;
          else if (MODE == PERIODIC) head = (ph >> c) & 1u;
          else head = (sh_heads[(rel0 + c) >> 5] >> ((rel0 + c) & 31)) & 1u;
          e[c] = head ? O::id() : (c == 0 ? prev : y[c - 1]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) y[c] = e[c];
      }
      if (vec == 1 && g + 4 <= n) {
        x.x = __builtin_bit_cast(int, y[0]);
        x.y = __builtin_bit_cast(int, y[1]);
        x.z = __builtin_bit_cast(int, y[2]);
        x.w = __builtin_bit_cast(int, y[3]);
        __stcs(reinterpret_cast<int4 *>(out + eg), x);
      } else if (MAPPED == 1 && vec == 2 && g + 4 <= n) {   // descending: the last point's element first
        x.x = __builtin_bit_cast(int, y[3]);
        x.y = __builtin_bit_cast(int, y[2]);
        x.z = __builtin_bit_cast(int, y[1]);
        x.w = __builtin_bit_cast(int, y[0]);
        __stcs(reinterpret_cast<int4 *>(out + eg + addr.step(3)), x);
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (g + c < n) out[Addr::kAffine ? eg + addr.step(c) : addr(g + c)] = y[c];
      }
    }
  }
  if (MODE == CSR && args.sums && sh_any_end) {         // totals of non-empty segments ending here
    // the value at the segment's last element, from the staged tile
    T *sums = static_cast<T *>(args.sums);
    const int64_t tend = std::min<int64_t>(t0 + kTile, n);
    for (int64_t s = sh_seg0 + 1 + tid; s <= args.nseg; s += kThreads) {
      const int64_t b = args.offsets[s];
      if (b > tend) break;
      if (b <= t0 || args.offsets[s - 1] == b) continue;
      const int rel = (int)(b - 1 - t0);
      const int sub = rel / kSub, r2 = rel % kSub;
      const T *v = reinterpret_cast<const T *>(ring + sub * kStageBytes + chunk_off(r2 / 4));
      T y = v[r2 % 4];
      if ((sh_need[sub * kThreads + r2 / kItems] >> (r2 % kItems)) & 1u) y = O::apply(y, pre);
      sums[s - 1] = y;
    }
  }
}

// ---- the scan through a lowered map, and the arg operators ----------------
// One CTA per tile of kMapTile logical points (tiles in ticket order).  The
// CTA loads point g of the tile from in[map(g)] (striped, so a warp reads
// consecutive points), stages the tile in shared memory, scans it (each
// thread 16 consecutive points, warp shuffles, warp totals), publishes and
// looks back as above, and stores point g's result to out[map(g)].  With
// the identity map this is a plain (or segmented) scan; with any other
// lowered map it scans a view in one pass, gathering in its loads and
// scattering in its stores.  Element states are values, or for the arg
// operators (value, position) pairs whose stored result is the base-array
// index of the position.
constexpr int kMapThreads = 256, kMapItems = 16, kMapTile = kMapThreads * kMapItems;
static_assert(kMapTile == kScanSubTile, "workspace tiles count kScanSubTile elements");

// Element-state layer of the map kernel for the value operators (the state
// is the value; make() takes the value and its element index) ...
template <class T, class O>
struct ValueStates {
  using Op = O;
  using E = T;
  using C = typename O::C;
  __device__ static E make(T x, int64_t) { return x; }
  __device__ static E eid() { return O::id(); }
  __device__ static E ecomb(E a, E b) { return O::comb(a, b); }   // a before b
  __device__ static E shfl_up(E e, int off) { return __shfl_up_sync(0xffffffffu, e, off); }
  __device__ static E shfl(E e, int src) { return __shfl_sync(0xffffffffu, e, src); }
  __device__ static E apply(E e, const C &c) { return O::apply(e, c); }
  __device__ static E of_carry(const C &c) { return O::apply(O::id(), c); }
  __device__ static C carry(E e) { return C::of(e); }
  __device__ static uint32_t out_bits(E e, const MapArgs &) { return __builtin_bit_cast(uint32_t, e); }
};

// ... and for the arg operators: (value, element index in the base array),
// index -1 = none; the better of two states by arg_better (ties: the smaller
// element index, whatever order the map visits the elements in).
template <class T, bool MAX>
struct ArgStates {
  struct E {
    T v;
    int32_t i;                      // element index, -1: none
  };
  struct Op;
  struct C {
    E e;
    __device__ static C zero() { return {{T(0), -1}}; }
    __device__ static C of(E x) { return {x}; }
    __device__ C plus(const C &o) const;
    __device__ C shfl_down(int off) const {
      return {{__shfl_down_sync(0xffffffffu, e.v, off), __shfl_down_sync(0xffffffffu, e.i, off)}};
    }
  };
  struct Op {
    using C = ArgStates::C;
    // 30 bits of element index: 0x3FFFFFFF stands for none.
    __device__ static unsigned long long pack(unsigned long long st, const C &c) {
      const uint32_t pos = c.e.i < 0 ? 0x3FFFFFFFu : (uint32_t)c.e.i;
      return (st << 62) | ((unsigned long long)pos << 32) | (unsigned long long)__builtin_bit_cast(uint32_t, c.e.v);
    }
    __device__ static C unpack(unsigned long long w) {
      const uint32_t pos = (uint32_t)(w >> 32) & 0x3FFFFFFFu;
      return {{__builtin_bit_cast(T, (uint32_t)w), pos == 0x3FFFFFFFu ? -1 : (int32_t)pos}};
    }
  };
  __device__ static E better(E a, E b) { return arg_better<T, MAX>(a.v, a.i, b.v, b.i) ? a : b; }
  __device__ static E make(T x, int64_t elem) { return {x, (int32_t)elem}; }
  __device__ static E eid() { return {T(0), -1}; }
  __device__ static E ecomb(E a, E b) { return better(a, b); }
  __device__ static E shfl_up(E e, int off) {
    return {__shfl_up_sync(0xffffffffu, e.v, off), __shfl_up_sync(0xffffffffu, e.i, off)};
  }
  __device__ static E shfl(E e, int src) {
    return {__shfl_sync(0xffffffffu, e.v, src), __shfl_sync(0xffffffffu, e.i, src)};
  }
  __device__ static E apply(E e, const C &c) { return better(c.e, e); }
  __device__ static E of_carry(const C &c) { return c.e; }
  __device__ static C carry(E e) { return {e}; }
  __device__ static uint32_t out_bits(E e, const MapArgs &) { return (uint32_t)e.i; }
};
template <class T, bool MAX>
__device__ __forceinline__ typename ArgStates<T, MAX>::C ArgStates<T, MAX>::C::plus(const C &o) const {
  return {ArgStates<T, MAX>::better(e, o.e)};
}

// The tile in shared memory.  4-byte states use the look-back scan's
// layout: 16-byte chunks in XOR-swizzled slots (chunk_off), conflict-free
// for a warp's striped chunks, a warp's 32 consecutive points and each
// thread's 4 consecutive chunks.  8-byte states (the arg operators) take one
// padding slot per 16.
template <class E>
struct MapTileSmem {
  static constexpr int kBytes = sizeof(E) == 4 ? kMapTile * 4 : (kMapTile + kMapTile / 16) * 8;
  __device__ static E *at(unsigned char *t, int r) {
    if constexpr (sizeof(E) == 4) return reinterpret_cast<E *>(t + chunk_off(r >> 2) + 4 * (r & 3));
    else return reinterpret_cast<E *>(t) + (r + (r >> 4));
  }
};

// Compute warps only (the look-back warp has left).
__device__ __forceinline__ void map_compute_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kMapThreads) : "memory"); }

// Warps 0..7 load the tile through the map (128-bit chunks where the map's
// inner dim is unit-stride: vec), stage it, scan it and store it; warp 8
// looks back from the start, while the loads are in flight.  mode: PLAIN,
// PERIODIC or CSR; excl: the exclusive form.
template <class T, class S>
__global__ void __launch_bounds__(kMapThreads + 32) scan_map_kernel(const T *__restrict__ in, uint32_t *__restrict__ out,
                                                                    const MapArgs m, ScanArgs args, ScanWs *ws,
                                                                    TileState *states, int mode, int excl) {
  using E = typename S::E;
  using O = typename S::Op;
  using CT = typename S::C;
  using SM = MapTileSmem<E>;
  constexpr bool kVec4 = sizeof(E) == 4;
  __shared__ __align__(128) unsigned char tile_smem[SM::kBytes];
  __shared__ unsigned sh_heads[kMapTile / 32];
  __shared__ E sh_wval[kMapThreads / 32];
  __shared__ int sh_wflag[kMapThreads / 32];
  __shared__ E sh_agg;
  __shared__ int sh_aggf;
  __shared__ CT sh_prefix;
  __shared__ int64_t sh_tile, sh_seg0;
  __shared__ int sh_ok;
  __shared__ volatile int sh_go;                       // the tile's inputs have landed: start polling

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    sh_tile = atomicAdd(&ws->ticket, 1u);
    sh_go = 0;
  }
  if (mode == CSR)
    for (int i = tid; i < kMapTile / 32; i += kMapThreads + 32) sh_heads[i] = 0u;
  if (warp < kMapThreads / 32) {                       // the guessed tile into L2 (as scan_kernel)
    const int64_t g = int64_t(blockIdx.x) * kMapTile + 16 * int64_t(tid);
    if (g < args.n) asm volatile("prefetch.global.L2 [%0];" ::"l"(in + map_elem(m, g)));
  }
  __syncthreads();
  const int64_t tile = sh_tile, t0 = tile * kMapTile, n = args.n;
  const int64_t tend = min(t0 + kMapTile, n);
  const bool stall = args.debug && tile == 1;

  if (warp == kMapThreads / 32) {
    // ---- look-back warp: the prefix of everything before t0
    bool first_head = tile == 0;
    if (mode == PERIODIC) first_head = first_head || t0 % args.period == 0;
    if (mode == CSR) first_head = first_head || args.offsets[find_segment(args.offsets, args.nseg, t0)] == t0;
    CT prefix = CT::zero();
    bool ok = true;
    if (!first_head) {
      // Predecessors publish about when this tile's own loads land; polls
      // before that only load the tile states (bounded wait).
      for (unsigned i = 0; i < kGoSpins && !sh_go; ++i) __nanosleep(64);
      ok = look_back<O>(states, tile, ws, args.debug ? kDebugBudgetCycles : kBudgetCycles, prefix);
    }
    if (lane == 0) {
      sh_prefix = prefix;
      sh_ok = ok ? 1 : 0;
    }
    __syncthreads();                                   // (S) the tile's aggregate is known
    if (ok && lane == 0 && !stall && tile != 0 && !sh_aggf)
      publish<O>(&states[tile], kStatIncl, prefix.plus(S::carry(sh_agg)));
    return;
  }

  unsigned char *tsm = tile_smem;
  const bool vec = args.vec != 0;
  // ---- loads through the map
  bool done = false;
  if constexpr (kVec4) {
    if (vec) {                                         // chunk c = points 4c .. 4c + 3
      done = true;
#pragma unroll
    for (int q = 0; q < kMapTile / 4 / kMapThreads; ++q) {
      const int c = q * kMapThreads + tid;
      const int64_t g = t0 + 4 * int64_t(c);
      int4 x;
      if (g + 4 <= n) {
        x = __ldcs(reinterpret_cast<const int4 *>(in + map_elem(m, g)));
      } else {
        E e[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) e[k] = g + k < n ? S::make(in[map_elem(m, g + k)], 0) : S::eid();
        x = make_int4(__builtin_bit_cast(int, e[0]), __builtin_bit_cast(int, e[1]), __builtin_bit_cast(int, e[2]),
                      __builtin_bit_cast(int, e[3]));
      }
      *reinterpret_cast<int4 *>(tsm + chunk_off(c)) = x;
    }
    }
  }
  if (!done) {
#pragma unroll
    for (int j = 0; j < kMapItems; ++j) {
      const int r = j * kMapThreads + tid;
      const int64_t g = t0 + r;
      E x = S::eid();
      if (g < n) {
        const int64_t e = map_elem(m, g);
        x = S::make(in[e], e);
      }
      *SM::at(tsm, r) = x;
    }
  }
  // ---- segment heads (CSR): boundaries offsets[q] in (t0, tend), and t0
  if (mode == CSR) {
    if (warp == 0) {
      const int64_t s0 = find_segment(args.offsets, args.nseg, t0);
      if (lane == 0) {
        sh_seg0 = s0;
        if (args.offsets[s0] == t0) atomicOr(&sh_heads[0], 1u);
      }
    }
    map_compute_bar();
    for (int64_t q = sh_seg0 + 1 + tid; q <= args.nseg; q += kMapThreads) {
      const int64_t b = args.offsets[q];
      if (b >= tend) break;
      if (b > t0) atomicOr(&sh_heads[(b - t0) >> 5], 1u << ((b - t0) & 31));
    }
  }
  map_compute_bar();
  if (tid == 0) sh_go = 1;
  auto is_head = [&](int r) -> bool {
    const int64_t g = t0 + r;
    if (mode == PLAIN) return g == 0;
    if (mode == PERIODIC) return g % args.period == 0;
    return (sh_heads[r >> 5] >> (r & 31)) & 1u;
  };

  // ---- scan of the tile: 16 consecutive points per thread
  const int r0 = tid * kMapItems;
  E v[kMapItems];
  if constexpr (kVec4) {
#pragma unroll
    for (int q = 0; q < kMapItems / 4; ++q) {
      const int4 x = *reinterpret_cast<const int4 *>(tsm + chunk_off((kMapItems / 4) * tid + q));
      v[4 * q] = __builtin_bit_cast(E, x.x);
      v[4 * q + 1] = __builtin_bit_cast(E, x.y);
      v[4 * q + 2] = __builtin_bit_cast(E, x.z);
      v[4 * q + 3] = __builtin_bit_cast(E, x.w);
    }
  } else {
#pragma unroll
    for (int i = 0; i < kMapItems; ++i) v[i] = *SM::at(tsm, r0 + i);
  }
  unsigned hm = 0u;
  if (mode == CSR) {
    hm = (sh_heads[r0 >> 5] >> (r0 & 31)) & 0xffffu;
  } else {
#pragma unroll
    for (int i = 0; i < kMapItems; ++i)
      if (is_head(r0 + i)) hm |= 1u << i;
  }
#pragma unroll
  for (int i = 1; i < kMapItems; ++i)
    if (!((hm >> i) & 1u)) v[i] = S::ecomb(v[i - 1], v[i]);
  int f = hm != 0u;
  E a = v[kMapItems - 1];
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {             // warp scan, segmented operator
    const E au = S::shfl_up(a, off);
    const int fu = __shfl_up_sync(0xffffffffu, f, off);
    if (lane >= off) {
      if (!f) a = S::ecomb(au, a);
      f |= fu;
    }
  }
  if (lane == 31) {
    sh_wval[warp] = a;
    sh_wflag[warp] = f;
  }
  E ex = S::shfl_up(a, 1);
  int exf = __shfl_up_sync(0xffffffffu, f, 1);
  if (lane == 0) {
    ex = S::eid();
    exf = 0;
  }
  map_compute_bar();
  if (warp == 0) {                                     // scan of the warp totals; publish
    constexpr int kW = kMapThreads / 32;
    E wa = lane < kW ? sh_wval[lane] : S::eid();
    int wf = lane < kW ? sh_wflag[lane] : 0;
#pragma unroll
    for (int off = 1; off < kW; off <<= 1) {
      const E au = S::shfl_up(wa, off);
      const int fu = __shfl_up_sync(0xffffffffu, wf, off);
      if (lane >= off) {
        if (!wf) wa = S::ecomb(au, wa);
        wf |= fu;
      }
    }
    E we = S::shfl_up(wa, 1);
    int wfe = __shfl_up_sync(0xffffffffu, wf, 1);
    if (lane == 0) {
      we = S::eid();
      wfe = 0;
    }
    const E agg = S::shfl(wa, kW - 1);
    const int aggf = __shfl_sync(0xffffffffu, wf, kW - 1);
    __syncwarp();
    if (lane < kW) {
      sh_wval[lane] = we;
      sh_wflag[lane] = wfe;
    }
    if (lane == 0) {
      sh_agg = agg;
      sh_aggf = aggf;
      // at once: the inclusive value when nothing before can change it
      // (tile 0, or a tile holding a segment head), else the tile total
      if (!stall) publish<O>(&states[tile], (tile == 0 || aggf) ? kStatIncl : kStatAgg, S::carry(agg));
    }
  }
  __syncthreads();                                     // (S) with the look-back warp
  if (!sh_ok) return;                                  // a wait gave up: write nothing
  {
    const E pv = sh_wval[warp];
    const int pf = sh_wflag[warp];
    if (!exf) ex = S::ecomb(pv, ex);
    exf |= pf;                                         // this thread's prefix within the tile
    const CT pre = sh_prefix;
#pragma unroll
    for (int i = 0; i < kMapItems; ++i)
      if ((hm & ((2u << i) - 1u)) == 0u) {             // no head in this thread up to item i
        E x = S::ecomb(ex, v[i]);
        v[i] = exf ? x : S::apply(x, pre);
      }
  }
  if constexpr (kVec4) {                               // each thread rewrites only its own chunks
#pragma unroll
    for (int q = 0; q < kMapItems / 4; ++q)
      *reinterpret_cast<int4 *>(tsm + chunk_off((kMapItems / 4) * tid + q)) =
          make_int4(__builtin_bit_cast(int, v[4 * q]), __builtin_bit_cast(int, v[4 * q + 1]),
                    __builtin_bit_cast(int, v[4 * q + 2]), __builtin_bit_cast(int, v[4 * q + 3]));
  } else {
#pragma unroll
    for (int i = 0; i < kMapItems; ++i) *SM::at(tsm, r0 + i) = v[i];
  }
  map_compute_bar();

  // ---- stores through the map (the exclusive form shifts by one)
  const E before = S::of_carry(sh_prefix);             // everything before the tile
  auto result = [&](int r) -> E {
    if (!excl) return *SM::at(tsm, r);
    return is_head(r) ? S::eid() : (r == 0 ? before : *SM::at(tsm, r - 1));
  };
  bool stored = false;
  if constexpr (kVec4) {
    if (vec) {
      stored = true;
#pragma unroll
    for (int q = 0; q < kMapTile / 4 / kMapThreads; ++q) {
      const int c = q * kMapThreads + tid;
      const int64_t g = t0 + 4 * int64_t(c);
      if (g >= n) break;
      uint32_t w[4];
      if (!excl) {
        const int4 x = *reinterpret_cast<const int4 *>(tsm + chunk_off(c));
        w[0] = (uint32_t)x.x; w[1] = (uint32_t)x.y; w[2] = (uint32_t)x.z; w[3] = (uint32_t)x.w;
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] = S::out_bits(result(4 * c + k), m);
      }
      if (g + 4 <= n) {
        __stcs(reinterpret_cast<int4 *>(out + map_elem(m, g)), make_int4((int)w[0], (int)w[1], (int)w[2], (int)w[3]));
      } else {
        for (int k = 0; k < 4 && g + k < n; ++k) out[map_elem(m, g + k)] = w[k];
      }
    }
    }
  }
  if (!stored) {
#pragma unroll
    for (int j = 0; j < kMapItems; ++j) {
      const int r = j * kMapThreads + tid;
      const int64_t g = t0 + r;
      if (g >= n) break;
      out[map_elem(m, g)] = S::out_bits(result(r), m);
    }
  }
  // ---- CSR: totals of the non-empty segments that end in this tile (the
  // empty ones hold the identity already)
  if (mode == CSR && args.sums) {
    uint32_t *sums = static_cast<uint32_t *>(args.sums);
    for (int64_t q = sh_seg0 + 1 + tid; q <= args.nseg; q += kMapThreads) {
      const int64_t b = args.offsets[q];
      if (b > tend) break;
      if (b <= t0 || args.offsets[q - 1] == b) continue;
      sums[q - 1] = S::out_bits(*SM::at(tsm, (int)(b - 1 - t0)), m);
    }
  }
}

// ---- the arg operators over contiguous runs ---------------------------------
// An element (x, index) as one 64-bit key whose unsigned maximum is the
// arg-maximum (arg-minimum): the high word is an order-preserving code of x
// (for the minimum, of -x in effect), with every NaN at 0 and -0 read as +0;
// the low word is ~index, so that among equal codes the smaller index wins.
// Key 0 is "no element".  A real key is never 0: ~index has its two top bits
// set for every index below 2^30.
template <class T, bool MAX>
__device__ __forceinline__ uint32_t order_code(T x) {
  if constexpr (std::is_same<T, float>::value) {
    const uint32_t u = __float_as_uint(__fadd_rn(x, 0.0f));   // -0 + 0 = +0; every other x kept
    const uint32_t k = u ^ (uint32_t(int32_t(u) >> 31) | 0x80000000u);   // monotone in x
    return x != x ? 0u : (MAX ? k : ~k);                // NaN: below every number
  } else {
    const uint32_t k = uint32_t(x) ^ 0x80000000u;       // monotone in x
    return MAX ? k : ~k;
  }
}

// The value a (non-zero) order code stands for: order_code inverted, -0
// coming back as +0.
template <class T, bool MAX>
__device__ __forceinline__ T code_value(uint32_t code) {
  const uint32_t k = MAX ? code : ~code;
  if constexpr (std::is_same<T, float>::value) {
    return __uint_as_float((k & 0x80000000u) ? (k ^ 0x80000000u) : ~k);
  } else {
    return T(k ^ 0x80000000u);
  }
}

// The better of two values under the arg operator's order, NaN losing to
// every number (fmaxf / fminf return the other operand); which of two equal
// values (+0, -0) comes back does not matter to the callers.
template <class T, bool MAX>
__device__ __forceinline__ T value_better(T a, T b) {
  if constexpr (std::is_same<T, float>::value) return MAX ? fmaxf(a, b) : fminf(a, b);
  else return MAX ? max(a, b) : min(a, b);
}

template <class T, bool MAX>
struct ArgKeys {
  using E = unsigned long long;
  struct C {
    E k;
    __device__ static C zero() { return {0ull}; }
    __device__ static C of(E x) { return {x}; }
    __device__ C plus(const C &o) const { return {k > o.k ? k : o.k}; }
    __device__ C shfl_down(int off) const {
      return {(E)__shfl_down_sync(0xffffffffu, (long long)k, off)};
    }
  };
  // In a 62-bit tile state: the code and the low 30 bits of ~index (the top
  // two are 1 for every real key); all 62 bits 0 is "no element".
  struct Op {
    using C = ArgKeys::C;
    __device__ static unsigned long long pack(unsigned long long st, const C &c) {
      return (st << 62) | ((c.k >> 32) << 30) | (c.k & 0x3FFFFFFFull);
    }
    __device__ static C unpack(unsigned long long w) {
      const unsigned long long code = (w >> 30) & 0xFFFFFFFFull, low = w & 0x3FFFFFFFull;
      if (code == 0 && low == 0) return {0ull};
      return {(code << 32) | 0xC0000000ull | low};
    }
  };
  __device__ static E eid() { return 0ull; }
  __device__ static E ecomb(E a, E b) { return a > b ? a : b; }
  __device__ static E shfl_up(E e, int off) { return (E)__shfl_up_sync(0xffffffffu, (long long)e, off); }
  __device__ static E shfl(E e, int src) { return (E)__shfl_sync(0xffffffffu, (long long)e, src); }
  __device__ static C carry(E e) { return {e}; }
};

// The look-back scan's pipeline (ticket with the guessed tile prefetched,
// cp.async into the swizzled stages, a look-back warp) over tiles of two
// 4096-point sub-tiles, for the arg-maximum / arg-minimum: point g is element
// idx_base + g.  Two passes over the staged tile.  The first reduces each
// thread's 16 points of each sub-tile to its best after the last segment head
// among them -- on the values (a NaN-losing max / min, then the first
// position holding it) with one 32-bit order code for the result -- and
// scans the threads' results, as 64-bit keys, over the whole tile at once
// (warp shuffles, then every warp scans the 16 warp totals itself).  Once the
// look-back prefix is known the second pass walks each thread's points from
// its start state, one value comparison a point (a thread whose start beats
// all its points writes the start's index 16 times), and each warp stores its
// 512 indices (inclusive or exclusive) as whole rows through its own slots
// of the stage.  The tile state carries ArgKeys.
// SUBS sub-tiles a tile; PIPE: pass 1 takes each sub-tile as it lands (one
// barrier each, the look-back released at the first) instead of all at once;
// MINB CTAs a SM (registers capped to fit; three for PERIODIC, whose head
// masks would spill at four).  Measured on 2^28 FP32: two
// pipelined sub-tiles at four CTAs a SM 0.43-0.45 ms; three CTAs 0.48,
// five the same as four (with spills), six 0.52; four sub-tiles 0.54.
constexpr int kArgSub = 2;
constexpr bool kArgPipe = true;
constexpr int kArgBlocksPerSM = 4;
constexpr int kArgTile = kSub * kArgSub;
constexpr int kArgSmem = kArgSub * kStageBytes;
static_assert(kItems == 16, "a thread's points are one 16-bit head mask");

// MAPPED (the map's dims, 1 or 2; 0: a contiguous run): points are read and
// written through the lowered map m, and point g is element m(g) of the base
// array; there the element indices need not grow with g, so the scan keeps
// every point's full key (code, ~index) instead of its position.
template <class T, bool MAX, int MODE, bool EXCL, int SUBS = kArgSub, bool PIPE = kArgPipe,
          int MINB = (MODE == PERIODIC ? 3 : kArgBlocksPerSM), int MAPPED = 0>
__global__ void __launch_bounds__(kThreads + 32, MINB) scan_arg_kernel(const T *in, int32_t *out, ScanArgs args,
                                                                    int64_t idx_base, ScanWs *ws,
                                                                    TileState *states,
                                                                    const __grid_constant__ MapArgs m) {
  using S = ArgKeys<T, MAX>;
  using E = typename S::E;
  using O = typename S::Op;
  using CT = typename S::C;
  static_assert(SUBS * kWarps <= 32 && SUBS <= 4, "one lane a warp total");
  static_assert(MAPPED == 0 || MODE != CSR, "the CSR call scans contiguous runs");
  constexpr int kTile = kSub * SUBS;
  constexpr int kTotals = SUBS * kWarps;           // warp totals in tile order
  extern __shared__ __align__(128) unsigned char ring[];   // SUBS stages
  __shared__ int64_t sh_tile, sh_seg0;
  __shared__ E sh_wval[kTotals];
  __shared__ int sh_wflag[kTotals];
  __shared__ E sh_carry;                // the tile's aggregate
  __shared__ int sh_carry_flag;         // a segment starts in the tile
  __shared__ CT sh_prefix;
  __shared__ int sh_ok;
  __shared__ unsigned sh_heads[MODE == CSR ? kTile / 32 : 1];   // one bit a point: a segment starts there
  __shared__ volatile int sh_go;
  __shared__ int64_t sh_r0;             // PERIODIC: t0's position in its segment

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n = args.n;
  using Addr = typename std::conditional<MAPPED == 0, RunAddr, MapAddr<MAPPED == 2 ? 2 : 1>>::type;
  const int vec = MAPPED == 1 ? args.vec : (args.vec != 0 ? 1 : 0);   // 2 only through one-dim maps
  const Addr addr{m};
  // the key of a point of code c at g: (c, ~ element index)
  auto key_at = [&](uint32_t c, int64_t g) -> E { return ((E)c << 32) | (uint32_t)~(uint32_t)addr(g); };
  if (tid == 0) {
    sh_tile = atomicAdd(&ws->ticket, 1u);
    sh_go = 0;
  }
  if (MODE == CSR)
    for (int i = tid; i < kTile / 32; i += kThreads + 32) sh_heads[i] = 0u;
  if (warp < kWarps) {                                 // the guessed tile into L2 (as scan_kernel)
    const int64_t guess = int64_t(blockIdx.x) * kTile;
#pragma unroll
    for (int k = 0; k < kTile / 32 / kThreads; ++k) {
      const int64_t g = guess + 32 * int64_t(k * kThreads + tid);
      if (g < n) asm volatile("prefetch.global.L2 [%0];" ::"l"(in + addr(g)));
    }
  }
  __syncthreads();
  const int64_t tile = sh_tile;
  const int64_t t0 = tile * kTile;
  const int64_t tend = std::min<int64_t>(t0 + kTile, n);
  const bool stall = args.debug && tile == 1;

  if (warp == kWarps) {
    // ---- look-back warp: the prefix of everything before t0
    bool first_is_head = tile == 0;
    if (MODE == PERIODIC) first_is_head = first_is_head || (t0 % args.period == 0);
    if (MODE == CSR) first_is_head = first_is_head || args.offsets[find_segment(args.offsets, args.nseg, t0)] == t0;
    CT prefix = CT::zero();
    bool ok = true;
    if (!first_is_head) {
      for (unsigned i = 0; i < kGoSpins && !sh_go; ++i) __nanosleep(64);
      ok = look_back<O>(states, tile, ws, args.debug ? kDebugBudgetCycles : kBudgetCycles, prefix);
    }
    if (lane == 0) {
      sh_prefix = prefix;
      sh_ok = ok ? 1 : 0;
    }
    __syncthreads();                                    // (S) the tile's state is known
    if (ok && lane == 0 && !stall && tile != 0 && !sh_carry_flag)
      publish<O>(&states[tile], kStatIncl, prefix.plus(S::carry(sh_carry)));
    return;
  }

  // ---- compute warps
#pragma unroll
  for (int s = 0; s < SUBS; ++s) {
    load_sub<T, MAPPED == 1>(ring + s * kStageBytes, in, t0 + int64_t(s) * kSub, n, vec, addr);
    cp_async_commit();
  }
  if (MODE == CSR) {                                   // segment heads: offsets[q] in (t0, tend), and t0
    if (warp == 0) {
      const int64_t s0 = find_segment(args.offsets, args.nseg, t0);
      if (lane == 0) {
        sh_seg0 = s0;
        if (args.offsets[s0] == t0 || t0 == 0) atomicOr(&sh_heads[0], 1u);
      }
    }
    compute_bar();
    for (int64_t q = sh_seg0 + 1 + tid; q <= args.nseg; q += kThreads) {
      const int64_t b = args.offsets[q];
      if (b >= tend) break;
      if (b > t0) atomicOr(&sh_heads[(b - t0) >> 5], 1u << ((b - t0) & 31));
    }
  }
  // this thread's absolute index of its first point in sub-tile 0 (below 2^30)
  const int32_t ibase = int32_t(idx_base + t0) + tid * kItems;
  if (MODE == PERIODIC && tid == 0) sh_r0 = t0 % args.period;   // one 64-bit division a tile
  if (!PIPE) {
    cp_async_wait<0>();
    compute_bar();                                      // the tile and its heads are visible
    if (tid == 0) sh_go = 1;
  }

  // ---- pass 1: order codes in place; per sub-tile the thread's aggregate
  // and its warp-exclusive prefix
  E ex[SUBS];
  int exf[SUBS];
  unsigned hmq[SUBS];
  uint32_t tmax[SUBS];                                  // the best code after the thread's last head
  E tkey[SUBS];                                         // MAPPED: the best key after it
#pragma unroll
  for (int s = 0; s < SUBS; ++s) {
    unsigned char *st = ring + s * kStageBytes;
    if (PIPE) {
      cp_async_wait_dyn(SUBS - 1 - s);
      compute_bar();                                    // sub-tile s (and the heads) visible
      if (s == 0 && tid == 0) sh_go = 1;
    }
    const int rel0 = s * kSub + tid * kItems;
    const int64_t g0 = t0 + rel0;
    const int64_t lim64 = n - g0;
    const int lim = lim64 >= kItems ? kItems : (lim64 > 0 ? int(lim64) : 0);
    unsigned hm = 0u;
    if (MODE == PLAIN) {
      hm = g0 == 0 ? 1u : 0u;
    } else if (MODE == PERIODIC) {
      hm = seg_heads<kItems>(seg_pos<kTile>(sh_r0, rel0, args), args.period);
    } else {
      hm = (sh_heads[rel0 >> 5] >> (rel0 & 31)) & 0xffffu;
    }
    hmq[s] = hm;
    // a contiguous scan leaves the values in the stage (pass 2 compares values);
    // a scan through a map replaces them by their order codes
    T xv[kItems];
    uint32_t c[kItems];
#pragma unroll
    for (int q = 0; q < kItems / 4; ++q) {
      int4 *p = reinterpret_cast<int4 *>(st + chunk_off((kItems / 4) * tid + q));
      const int4 x = chunk_in_order<MAPPED == 1>(*p, vec);
      xv[4 * q + 0] = __builtin_bit_cast(T, x.x);
      xv[4 * q + 1] = __builtin_bit_cast(T, x.y);
      xv[4 * q + 2] = __builtin_bit_cast(T, x.z);
      xv[4 * q + 3] = __builtin_bit_cast(T, x.w);
      if constexpr (MAPPED != 0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) c[4 * q + e] = order_code<T, MAX>(xv[4 * q + e]);
        *p = make_int4(int(c[4 * q]), int(c[4 * q + 1]), int(c[4 * q + 2]), int(c[4 * q + 3]));
      }
    }
    E a;
    if constexpr (MAPPED == 0) {
      // the best code after the thread's last head, its first position on ties
      uint32_t best = 0u;
      int pos = -1;
      if (hm == 0u && lim == kItems) {                  // the extreme value, then its first position
        T mv = xv[0];
#pragma unroll
        for (int i = 1; i < kItems; ++i) mv = value_better<T, MAX>(mv, xv[i]);   // NaN loses
        pos = kItems - 1;
#pragma unroll
        for (int i = kItems - 2; i >= 0; --i) pos = xv[i] == mv ? i : pos;      // -0 == +0
        if constexpr (std::is_same<T, float>::value)
          if (mv != mv) pos = 0;                        // all NaN: the first
        best = order_code<T, MAX>(mv);
      } else {
#pragma unroll
        for (int i = 0; i < kItems; ++i)
          if (i < lim) {
            const uint32_t ci = order_code<T, MAX>(xv[i]);
            if (((hm >> i) & 1u) || pos < 0 || ci > best) {
              best = ci;
              pos = i;
            }
          }
      }
      tmax[s] = best;
      a = pos < 0 ? S::eid() : ((E)best << 32) | (uint32_t)~(uint32_t)(ibase + s * kSub + pos);
    } else {
      // the largest key after the thread's last head
      E kb = S::eid();
      if (hm == 0u && lim == kItems) {
#pragma unroll
        for (int i = 0; i < kItems; ++i) kb = S::ecomb(kb, key_at(c[i], g0 + i));
      } else {
#pragma unroll
        for (int i = 0; i < kItems; ++i)
          if (i < lim) {
            const E ki = key_at(c[i], g0 + i);
            kb = ((hm >> i) & 1u) ? ki : S::ecomb(kb, ki);
          }
      }
      tkey[s] = kb;
      a = kb;
    }
    int f = hm != 0u;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {           // warp scan, segmented operator
      const E au = S::shfl_up(a, off);
      const int fu = __shfl_up_sync(0xffffffffu, f, off);
      if (lane >= off) {
        if (!f) a = S::ecomb(au, a);
        f |= fu;
      }
    }
    if (lane == 31) {
      sh_wval[s * kWarps + warp] = a;
      sh_wflag[s * kWarps + warp] = f;
    }
    ex[s] = S::shfl_up(a, 1);
    exf[s] = __shfl_up_sync(0xffffffffu, f, 1);
    if (lane == 0) {
      ex[s] = S::eid();
      exf[s] = 0;
    }
  }
  compute_bar();
  // every warp scans the warp totals of the whole tile (sub-tile 0's warps, then sub-tile 1's)
  E wa = lane < kTotals ? sh_wval[lane] : S::eid();
  int wf = lane < kTotals ? sh_wflag[lane] : 0;
#pragma unroll
  for (int off = 1; off < kTotals; off <<= 1) {
    const E au = S::shfl_up(wa, off);
    const int fu = __shfl_up_sync(0xffffffffu, wf, off);
    if (lane >= off) {
      if (!wf) wa = S::ecomb(au, wa);
      wf |= fu;
    }
  }
  const E tot = S::shfl(wa, kTotals - 1);
  const int totf = __shfl_sync(0xffffffffu, wf, kTotals - 1);
  E we = S::shfl_up(wa, 1);
  int wfe = __shfl_up_sync(0xffffffffu, wf, 1);
  if (lane == 0) {
    we = S::eid();
    wfe = 0;
  }
  E start[SUBS];                                     // in-tile state before the thread's points
  int sflag[SUBS];                                   // a head precedes them in the tile
#pragma unroll
  for (int s = 0; s < SUBS; ++s) {
    const E pv = S::shfl(we, s * kWarps + warp);
    const int pf = __shfl_sync(0xffffffffu, wfe, s * kWarps + warp);
    start[s] = exf[s] ? ex[s] : S::ecomb(pv, ex[s]);    // (pf, pv) then (exf, ex)
    sflag[s] = exf[s] | pf;
  }
  if (tid == 0) {
    if (!stall) publish<O>(&states[tile], (tile == 0 || totf) ? kStatIncl : kStatAgg, S::carry(tot));
    sh_carry = tot;
    sh_carry_flag = totf;
  }
  __syncthreads();                                      // (S) with the look-back warp
  if (!sh_ok) return;
  const E pre = sh_prefix.k;

  // ---- pass 2: each thread's points from its start state.  Where a CSR
  // call wants its segment totals, the inclusive indices stay in the stage
  // and each thread stores its 16 results itself; otherwise the results take
  // the place of the thread's codes and each warp stores its 512 points as
  // whole rows.
  const bool keep_incl = MODE == CSR && args.sums != nullptr;
#pragma unroll
  for (int s = 0; s < SUBS; ++s) {
    unsigned char *st = ring + s * kStageBytes;
    const E e0 = sflag[s] ? start[s] : S::ecomb(pre, start[s]);
    uint32_t best = uint32_t(e0 >> 32);
    int32_t idx = int32_t(~uint32_t(e0));               // "no element": code 0, index -1
    const int32_t ib = ibase + s * kSub;
    const unsigned hm = hmq[s];
    const int64_t g0 = t0 + s * kSub + tid * kItems;
    const int64_t lim64 = n - g0;
    const bool full = lim64 >= kItems;
    int32_t r[kItems];
    auto chunk = [&](int q) { return reinterpret_cast<int4 *>(st + chunk_off((kItems / 4) * tid + q)); };
    if constexpr (MAPPED != 0) {
      // the running key; a start key at least the thread's largest beats every point
      E cur = e0;
      if (hm == 0u && full && cur >= tkey[s]) {
#pragma unroll
        for (int i = 0; i < kItems; ++i) r[i] = int32_t(~uint32_t(cur));
      } else {
#pragma unroll
        for (int q = 0; q < kItems / 4; ++q) {
          const int4 x = *chunk(q);
          const uint32_t cs[4] = {uint32_t(x.x), uint32_t(x.y), uint32_t(x.z), uint32_t(x.w)};
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int i = 4 * q + c;
            const bool head = (hm >> i) & 1u;
            if (EXCL) r[i] = head ? -1 : int32_t(~uint32_t(cur));   // key 0: index -1
            if (i < lim64) {
              const E ki = key_at(cs[c], g0 + i);
              cur = head ? ki : S::ecomb(cur, ki);
            }
            if (!EXCL) r[i] = int32_t(~uint32_t(cur));
          }
        }
      }
    } else if (hm == 0u && full && idx >= 0 && best >= tmax[s]) {
      // the start state beats every point (on a tie it comes first)
#pragma unroll
      for (int i = 0; i < kItems; ++i) r[i] = idx;
      if (keep_incl)
#pragma unroll
        for (int q = 0; q < kItems / 4; ++q) *chunk(q) = make_int4(idx, idx, idx, idx);
    } else if (hm == 0u && full && (best != 0u || !std::is_same<T, float>::value)) {
      // compare values: the start state's value (a FP32 code 0 is a NaN, which
      // every number beats: the per-point codes below take that case)
      T bv = code_value<T, MAX>(best);
#pragma unroll
      for (int q = 0; q < kItems / 4; ++q) {
        const int4 x = *chunk(q);
        const T xs[4] = {__builtin_bit_cast(T, x.x), __builtin_bit_cast(T, x.y), __builtin_bit_cast(T, x.z),
                         __builtin_bit_cast(T, x.w)};
        int32_t in4[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int i = 4 * q + c;
          if (EXCL) r[i] = idx;
          const bool gt = MAX ? xs[c] > bv : xs[c] < bv;   // NaN and equal values lose
          bv = gt ? xs[c] : bv;
          idx = gt ? ib + i : idx;
          if (!EXCL) r[i] = idx;
          in4[c] = idx;
        }
        if (keep_incl) *chunk(q) = make_int4(in4[0], in4[1], in4[2], in4[3]);
      }
    } else {                                            // heads among the points, or the array's end
#pragma unroll
      for (int q = 0; q < kItems / 4; ++q) {
        int4 *p = chunk(q);
        const int4 x = *p;
        const uint32_t cs[4] = {order_code<T, MAX>(__builtin_bit_cast(T, x.x)),
                                order_code<T, MAX>(__builtin_bit_cast(T, x.y)),
                                order_code<T, MAX>(__builtin_bit_cast(T, x.z)),
                                order_code<T, MAX>(__builtin_bit_cast(T, x.w))};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int i = 4 * q + c;
          const bool head = (hm >> i) & 1u;
          if (EXCL) r[i] = head ? -1 : idx;
          if (i < lim64 && (head || idx < 0 || cs[c] > best)) {
            best = cs[c];
            idx = ib + i;
          }
          if (!EXCL) r[i] = idx;
          if (keep_incl) reinterpret_cast<int32_t *>(p)[c] = idx;   // inclusive, for the totals
        }
      }
    }
    if (keep_incl) {
      int32_t *o = out + g0;
      if (vec == 1 && full) {
#pragma unroll
        for (int q = 0; q < kItems / 4; ++q)
          __stcs(reinterpret_cast<int4 *>(o) + q, make_int4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]));
      } else {
#pragma unroll
        for (int i = 0; i < kItems; ++i)
          if (i < lim64) o[i] = r[i];
      }
    } else {
#pragma unroll
      for (int q = 0; q < kItems / 4; ++q) *chunk(q) = make_int4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
      __syncwarp();                                     // the warp's 512 results are in its own slots
      const int64_t gw = t0 + s * kSub + 4 * int64_t((kItems / 4) * 32 * warp + lane);   // chunk q = 0
      const int64_t e0 = Addr::kAffine ? addr(gw) : 0, de = Addr::kAffine ? addr.step(4 * 32) : 0;
#pragma unroll
      for (int q = 0; q < kItems / 4; ++q) {
        const int j = (kItems / 4) * 32 * warp + 32 * q + lane;   // chunk of the sub-tile
        const int4 v = *reinterpret_cast<const int4 *>(st + chunk_off(j));
        const int64_t g = t0 + s * kSub + 4 * int64_t(j);
        const int64_t eg = Addr::kAffine ? e0 + q * de : addr(g);   // the element of point g
        if (vec == 1 && g + 4 <= n) {
          __stcs(reinterpret_cast<int4 *>(out + eg), v);
        } else if (MAPPED == 1 && vec == 2 && g + 4 <= n) {   // descending: the last point's element first
          __stcs(reinterpret_cast<int4 *>(out + eg + addr.step(3)), make_int4(v.w, v.z, v.y, v.x));
        } else {
          const int32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (g + c < n) out[Addr::kAffine ? eg + addr.step(c) : addr(g + c)] = w[c];
        }
      }
    }
  }
  if (MODE == CSR && args.sums) {                       // totals of the non-empty segments ending here
    compute_bar();
    int32_t *sums = static_cast<int32_t *>(args.sums);
    for (int64_t q = sh_seg0 + 1 + tid; q <= args.nseg; q += kThreads) {
      const int64_t b = args.offsets[q];
      if (b > tend) break;
      if (b <= t0 || args.offsets[q - 1] == b) continue;
      const int rr = int(b - 1 - t0);
      sums[q - 1] = reinterpret_cast<const int32_t *>(ring + (rr / kSub) * kStageBytes +
                                                      chunk_off((rr % kSub) / 4))[rr % 4];
    }
  }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int kWsTile = kSub;   // workspace is sized for the smallest tile

// Schedule candidates: sub-tiles per tile (tile = 4096 x SUB elements; candidates.h).
static_assert(kSub == kScanSubTile, "the candidate table counts sub-tiles of this size");
static_assert(kSub * kScanSubCands[0] == kScanNoallocTile, "the no-alloc scan runs candidate 0");

template <class T, class O, int MODE, int SUB, bool EXCL, int MAPPED>
int32_t run_scan_t(const T *in, T *out, const ScanArgs &a, void *ws, size_t ws_bytes, cudaStream_t s,
                   const MapArgs &m) {
  constexpr int kTile = kSub * SUB;
  const int64_t ntiles = (a.n + kTile - 1) / kTile;
  if (ntiles == 0) return DESC_OK;
  const size_t need = align256(sizeof(ScanWs)) + size_t(ntiles) * sizeof(TileState);
  if (!ws || ws_bytes < need) return DESC_ERR_WORKSPACE;
  if (ntiles >= (int64_t(1) << 31)) return DESC_ERR_UNSUPPORTED;
  const int smem = SUB * kStageBytes;
  static std::atomic<unsigned long long> attr_devs{0};   // devices this kernel's attribute is set on
  int dev = 0;
  DESC_CUDA_TRY(cudaGetDevice(&dev));
  const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
  if (!(attr_devs.load(std::memory_order_acquire) & bit) || !bit) {
    DESC_CUDA_TRY(cudaFuncSetAttribute(scan_kernel<T, O, MODE, SUB, EXCL, MAPPED>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr_devs.fetch_or(bit, std::memory_order_release);
  }
  DESC_CUDA_TRY(cudaMemsetAsync(ws, 0, need, s));
  ScanWs *w = static_cast<ScanWs *>(ws);
  TileState *st = reinterpret_cast<TileState *>(static_cast<char *>(ws) + align256(sizeof(ScanWs)));
  scan_kernel<T, O, MODE, SUB, EXCL, MAPPED><<<(unsigned)ntiles, kThreads + 32, smem, s>>>(in, out, with_period(a), w,
                                                                                          st, m);
  DESC_CUDA_TRY(cudaGetLastError());
  return DESC_OK;
}

// The sum (every schedule candidate when inclusive and read directly, the
// default tile otherwise), the maximum and the minimum.
template <class T, int MODE, int MAPPED>
int32_t run_scan_basic(const T *in, T *out, const ScanArgs &a, void *ws, size_t ws_bytes, cudaStream_t s, int cand,
                       int32_t flags, const MapArgs &m) {
  const bool ex = (flags & DESC_EXCLUSIVE) != 0;
  auto go = [&](auto opv) -> int32_t {
    using O = decltype(opv);
    return ex ? run_scan_t<T, O, MODE, 4, true, MAPPED>(in, out, a, ws, ws_bytes, s, m)
              : run_scan_t<T, O, MODE, 4, false, MAPPED>(in, out, a, ws, ws_bytes, s, m);
  };
  switch (flags & kOperatorFlags) {
    case DESC_MAX: return go(ValOp<T, kMaxOp>{});
    case DESC_MIN: return go(ValOp<T, kMinOp>{});
    case 0: break;
    default: return DESC_ERR_INVALID_ARG;
  }
  if constexpr (MAPPED) {
    return go(SumOp<T>{});
  } else {
    if (ex) return go(SumOp<T>{});
    switch (kScanSubCands[(cand >= 0 && cand < kNumScanCands) ? cand : 0]) {
      case 1: return run_scan_t<T, SumOp<T>, MODE, 1, false, false>(in, out, a, ws, ws_bytes, s, m);
      case 2: return run_scan_t<T, SumOp<T>, MODE, 2, false, false>(in, out, a, ws, ws_bytes, s, m);
      default: return run_scan_t<T, SumOp<T>, MODE, 4, false, false>(in, out, a, ws, ws_bytes, s, m);
    }
  }
}

// The product (int32 and FP32) and the bitwise operators (int32), default tile.
template <class T, int MODE, int MAPPED>
int32_t run_scan_ops(const T *in, T *out, const ScanArgs &a, void *ws, size_t ws_bytes, cudaStream_t s,
                     int32_t flags, const MapArgs &m) {
  const bool ex = (flags & DESC_EXCLUSIVE) != 0;
  auto go = [&](auto opv) -> int32_t {
    using O = decltype(opv);
    return ex ? run_scan_t<T, O, MODE, 4, true, MAPPED>(in, out, a, ws, ws_bytes, s, m)
              : run_scan_t<T, O, MODE, 4, false, MAPPED>(in, out, a, ws, ws_bytes, s, m);
  };
  const int32_t op = flags & kOperatorFlags;
  if (op == DESC_PROD) return go(ValOp<T, kProdOp>{});
  if constexpr (std::is_same<T, int32_t>::value) {
    if (op == DESC_AND) return go(ValOp<T, kAndOp>{});
    if (op == DESC_OR) return go(ValOp<T, kOrOp>{});
    if (op == DESC_XOR) return go(ValOp<T, kXorOp>{});
  }
  return DESC_ERR_INVALID_ARG;
}

// ---- segments by groups of threads -----------------------------------------
// One group of G threads (a warp, or the whole CTA) per CSR segment, the
// groups striding over the segments.  The group walks its segment in steps of
// G x 4 points: each thread loads 4 consecutive points, scans them, the group
// scans the thread totals (shuffles; for a CTA also the warp totals in shared
// memory), applies the carry of the earlier steps and writes; the carry then
// takes in the step's total (compensated for FP32 sums).  No look-back and no
// workspace: suited to many short segments, where the tiles would hold many
// segment heads.
constexpr int kSegGroupThreads = 256, kSegItems = 4;

template <class T, class O, bool EXCL, int G>
__global__ void __launch_bounds__(kSegGroupThreads) seg_group_kernel(const T *__restrict__ in, T *__restrict__ out,
                                                                     const int64_t *__restrict__ offsets, int64_t nseg,
                                                                     T *__restrict__ sums) {
  using CT = typename O::C;
  constexpr int kGroups = kSegGroupThreads / G;
  constexpr int kStep = G * kSegItems;
  __shared__ T sh_w[kSegGroupThreads / 32];
  const int gl = threadIdx.x % G, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t sg = int64_t(blockIdx.x) * kGroups; sg < nseg; sg += int64_t(gridDim.x) * kGroups) {
    const int64_t s = sg + threadIdx.x / G;
    const bool live = s < nseg;                         // every thread takes part in the barriers
    const int64_t a = live ? offsets[s] : 0, b = live ? offsets[s + 1] : 0;
    CT carry = CT::zero();
    // with G = the CTA, every thread has the same segment and step count, so
    // the barriers inside the step are reached by all of them
    const int64_t nsteps = b > a ? (b - a + kStep - 1) / kStep : 0;
    for (int64_t k = 0; k < nsteps; ++k) {
      const int64_t p0 = a + k * kStep + int64_t(gl) * kSegItems;
      T v[kSegItems];
#pragma unroll
      for (int i = 0; i < kSegItems; ++i) v[i] = p0 + i < b ? in[p0 + i] : O::id();
#pragma unroll
      for (int i = 1; i < kSegItems; ++i) v[i] = O::comb(v[i - 1], v[i]);
      T t = v[kSegItems - 1];                           // inclusive scan of the thread totals
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const T u = __shfl_up_sync(0xffffffffu, t, off);
        if (lane >= off) t = O::comb(u, t);
      }
      T ex = __shfl_up_sync(0xffffffffu, t, 1);
      if (lane == 0) ex = O::id();
      T total = __shfl_sync(0xffffffffu, t, 31);
      if (G == kSegGroupThreads) {                      // across the warps of the CTA
        if (lane == 31) sh_w[warp] = t;
        __syncthreads();
        T wp = O::id();
        total = O::id();
#pragma unroll
        for (int w = 0; w < kSegGroupThreads / 32; ++w) {
          const T x = sh_w[w];
          if (w < warp) wp = O::comb(wp, x);
          total = O::comb(total, x);
        }
        ex = O::comb(wp, ex);
        __syncthreads();                                // sh_w is reused by the next step
      }
      // results: carry, then the thread's prefix within the step, then the item
      T prev = O::apply(ex, carry);                     // everything before this thread's first item
#pragma unroll
      for (int i = 0; i < kSegItems; ++i) {
        const T inc = O::apply(O::comb(ex, v[i]), carry);
        if (p0 + i < b) out[p0 + i] = EXCL ? prev : inc;
        prev = inc;
      }
      carry = carry.plus(CT::of(total));
    }
    if (live && gl == 0 && sums) sums[s] = O::apply(O::id(), carry);
  }
}

template <class T, class O, bool EXCL>
int32_t run_seg_group(const T *in, T *out, const int64_t *offsets, int64_t nseg, T *sums, int threads,
                      cudaStream_t s) {
  const int groups = kSegGroupThreads / threads;
  const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>((nseg + groups - 1) / groups, 152 * 16));
  if (threads == 32)
    seg_group_kernel<T, O, EXCL, 32><<<(unsigned)ctas, kSegGroupThreads, 0, s>>>(in, out, offsets, nseg, sums);
  else
    seg_group_kernel<T, O, EXCL, kSegGroupThreads><<<(unsigned)ctas, kSegGroupThreads, 0, s>>>(in, out, offsets,
                                                                                                 nseg, sums);
  DESC_CUDA_TRY(cudaGetLastError());
  return DESC_OK;
}


template <class T, class S>
struct StateTag {
  using Elem = T;
  using States = S;
};

// Calls f(StateTag<element type, state layer>{}) for the operator in flags.
template <class F>
int32_t with_states(int32_t dtype, int32_t flags, F &&f) {
  const int32_t op = flags & kOperatorFlags;
  if (dtype == DESC_I32) {
    using T = int32_t;
    switch (op) {
      case 0: return f(StateTag<T, ValueStates<T, SumOp<T>>>{});
      case DESC_MAX: return f(StateTag<T, ValueStates<T, ValOp<T, kMaxOp>>>{});
      case DESC_MIN: return f(StateTag<T, ValueStates<T, ValOp<T, kMinOp>>>{});
      case DESC_PROD: return f(StateTag<T, ValueStates<T, ValOp<T, kProdOp>>>{});
      case DESC_AND: return f(StateTag<T, ValueStates<T, ValOp<T, kAndOp>>>{});
      case DESC_OR: return f(StateTag<T, ValueStates<T, ValOp<T, kOrOp>>>{});
      case DESC_XOR: return f(StateTag<T, ValueStates<T, ValOp<T, kXorOp>>>{});
      case DESC_ARGMAX: return f(StateTag<T, ArgStates<T, true>>{});
      case DESC_ARGMIN: return f(StateTag<T, ArgStates<T, false>>{});
      default: return DESC_ERR_INVALID_ARG;
    }
  }
  using T = float;
  switch (op) {
    case 0: return f(StateTag<T, ValueStates<T, SumOp<T>>>{});
    case DESC_MAX: return f(StateTag<T, ValueStates<T, ValOp<T, kMaxOp>>>{});
    case DESC_MIN: return f(StateTag<T, ValueStates<T, ValOp<T, kMinOp>>>{});
    case DESC_PROD: return f(StateTag<T, ValueStates<T, ValOp<T, kProdOp>>>{});
    case DESC_ARGMAX: return f(StateTag<T, ArgStates<T, true>>{});
    case DESC_ARGMIN: return f(StateTag<T, ArgStates<T, false>>{});
    default: return DESC_ERR_INVALID_ARG;
  }
}


// The canonical map of nd dims (extent-1 dims dropped, neighbours merged)
// and its point count; nd == 0: the identity over `count` points.
int64_t build_map(int64_t off, const int64_t *ext, const int64_t *stride, int nd, int64_t count, MapArgs *m) {
  *m = MapArgs{};
  int64_t n = 1;
  for (int i = 0; i < nd; ++i) {
    m->ext[i] = ext[i];
    m->st[i] = stride[i];
    n *= ext[i];
  }
  if (nd == 0) n = count;
  m->off = off;
  int64_t *sets[1] = {m->st};
  m->nd = nd ? canon_dims(nd, m->ext, sets, 1) : 0;
  if (nd && m->nd == 0) {                              // a single point
    m->nd = 1;
    m->ext[0] = 1;
    m->st[0] = 0;
  }
  bool fast = n < (int64_t(1) << 32);
  for (int i = 0; i < m->nd; ++i) {
    fast = fast && m->ext[i] <= (int64_t(1) << 31);
    if (fast) m->div[i] = make_fastdiv((uint32_t)m->ext[i]);
  }
  m->fast = fast ? 1 : 0;
  return n;
}

// 128-bit accesses through the map: four consecutive points (from a multiple
// of 4) are four consecutive elements starting on a 16-byte boundary of in
// and out.
bool map_vec(const MapArgs &m, const void *in, const void *out) {
  bool vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0 && m.off % 4 == 0;
  if (m.nd >= 1) {
    vec = vec && m.st[m.nd - 1] == 1 && m.ext[m.nd - 1] % 4 == 0;
    for (int i = 0; i + 1 < m.nd; ++i) vec = vec && m.st[i] % 4 == 0;
  }
  return vec;
}


// 128-bit accesses to a reversed run: a one-dim map of stride -1 whose
// chunks of four points (from a multiple of 4) end on a 16-byte boundary.
bool map_descending(const MapArgs &m, const void *in, const void *out) {
  return ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0 && m.nd == 1 &&
         m.st[0] == -1 && (m.off + 1) % 4 == 0;
}

// The load mode of the look-back scans through a map (see load_sub).
int map_load_mode(const MapArgs &m, const void *in, const void *out) {
  return map_vec(m, in, out) ? 1 : (map_descending(m, in, out) ? 2 : 0);
}

// The look-back scan through a map of ND (1 or 2) canonical dims: every
// value operator, plain or per-level segments.
template <int ND>
int32_t run_scan_mapped_nd(int32_t dtype, const void *in, void *out, const MapArgs &m, int64_t n, int64_t period,
                           int32_t flags, void *ws, size_t ws_bytes, cudaStream_t s) {
  ScanArgs a{};
  a.n = n;
  a.period = period > 0 ? period : n;
  a.debug = (flags & DESC_DEBUG_STALL_TILE) ? 1 : 0;
  a.vec = map_load_mode(m, in, out);
  const bool periodic = a.period < n;
  const bool basic = !(flags & (DESC_PROD | DESC_AND | DESC_OR | DESC_XOR));
  auto go = [&](auto tag) -> int32_t {
    using T = decltype(tag);
    auto i = static_cast<const T *>(in);
    auto o = static_cast<T *>(out);
    if (basic)
      return periodic ? run_scan_basic<T, PERIODIC, ND>(i, o, a, ws, ws_bytes, s, -1, flags, m)
                      : run_scan_basic<T, PLAIN, ND>(i, o, a, ws, ws_bytes, s, -1, flags, m);
    return periodic ? run_scan_ops<T, PERIODIC, ND>(i, o, a, ws, ws_bytes, s, flags, m)
                    : run_scan_ops<T, PLAIN, ND>(i, o, a, ws, ws_bytes, s, flags, m);
  };
  return dtype == DESC_I32 ? go(int32_t(0)) : go(0.f);
}

// Reads and clears this translation unit's device status word.
int32_t take_status_word() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_scan_status, sizeof(int)) != cudaSuccess) return DESC_ERR_CUDA;
  if (v != 0 && cudaMemcpyToSymbol(g_scan_status, &z, sizeof(int)) != cudaSuccess) return DESC_ERR_CUDA;
  return v;
}

}  // namespace
}  // namespace desc
