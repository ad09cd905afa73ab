// Device helpers shared by the kernels of libdesc.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <type_traits>

#include "desc_internal.h"

namespace desc {

#define DESC_CUDA_TRY(expr)                        \
  do {                                             \
    cudaError_t _e = (expr);                       \
    if (_e != cudaSuccess) return DESC_ERR_CUDA;   \
  } while (0)

// Streaming 128-bit loads: evict-first in L1/L2 (each byte is read once).
__device__ __forceinline__ int4 ld_stream(const int4 *p) { return __ldcs(p); }
__device__ __forceinline__ float4 ld_stream(const float4 *p) { return __ldcs(p); }

// Error-free transformation of a sum (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Accumulators.  add1/add4 take elements, merge combines two partial
// accumulators, value() gives the final sum.
struct AccI32 {   // sum modulo 2^32
  static constexpr bool kIndexed = false;
  uint32_t s;
  __device__ void init() { s = 0u; }
  __device__ void add1(int32_t x) { s += (uint32_t)x; }
  __device__ void add4(int4 v) { s += ((uint32_t)v.x + (uint32_t)v.y) + ((uint32_t)v.z + (uint32_t)v.w); }
  __device__ void merge(const AccI32 &o) { s += o.s; }
  __device__ void shfl_merge(int off) { AccI32 o; o.s = __shfl_down_sync(0xffffffffu, s, off); merge(o); }
  __device__ uint2 pack() const { return make_uint2(s, 0u); }
  __device__ void unpack(uint2 v) { s = v.x; }
};

struct AccF32 {   // plain FP32 sum, pairwise inside each vector
  static constexpr bool kIndexed = false;
  float s;
  __device__ void init() { s = 0.f; }
  __device__ void add1(float x) { s = __fadd_rn(s, x); }
  __device__ void add4(float4 v) { s = __fadd_rn(s, __fadd_rn(__fadd_rn(v.x, v.y), __fadd_rn(v.z, v.w))); }
  __device__ void merge(const AccF32 &o) { s = __fadd_rn(s, o.s); }
  __device__ void shfl_merge(int off) { AccF32 o; o.s = __shfl_down_sync(0xffffffffu, s, off); merge(o); }
  __device__ uint2 pack() const { return make_uint2(__float_as_uint(s), 0u); }
  __device__ void unpack(uint2 v) { s = __uint_as_float(v.x); }
};

struct AccKahan {  // compensated FP32 sum (Neumaier's variant of Kahan summation)
  static constexpr bool kIndexed = false;
  float s, c;
  __device__ void init() { s = 0.f; c = 0.f; }
  __device__ void add1(float x) {
    const float t = __fadd_rn(s, x);
    if (fabsf(s) >= fabsf(x)) c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, t), x));
    else c = __fadd_rn(c, __fadd_rn(__fsub_rn(x, t), s));
    s = t;
  }
  __device__ void add4(float4 v) { add1(v.x); add1(v.y); add1(v.z); add1(v.w); }
  __device__ void merge(const AccKahan &o) {
    float t, e;
    two_sum(s, o.s, t, e);
    s = t;
    c = __fadd_rn(c, __fadd_rn(o.c, e));
  }
  __device__ void shfl_merge(int off) {
    AccKahan o;
    o.s = __shfl_down_sync(0xffffffffu, s, off);
    o.c = __shfl_down_sync(0xffffffffu, c, off);
    merge(o);
  }
  __device__ uint2 pack() const { return make_uint2(__float_as_uint(s), __float_as_uint(c)); }
  __device__ void unpack(uint2 v) { s = __uint_as_float(v.x); c = __uint_as_float(v.y); }
};

// Maximum / minimum (MAX true / false) of int32 or FP32; FP32 uses
// fmaxf / fminf, which ignore a NaN operand.
template <class T, bool MAX>
struct AccExt {
  static constexpr bool kIndexed = false;
  T v;
  __device__ static T ident() {
    if constexpr (std::is_same<T, float>::value) return MAX ? -__int_as_float(0x7f800000) : __int_as_float(0x7f800000);
    else return MAX ? INT32_MIN : INT32_MAX;
  }
  __device__ static T op(T a, T b) {
    if constexpr (std::is_same<T, float>::value) return MAX ? fmaxf(a, b) : fminf(a, b);
    else return MAX ? max(a, b) : min(a, b);
  }
  __device__ void init() { v = ident(); }
  __device__ void add1(T x) { v = op(v, x); }
  template <class V4>
  __device__ void add4(V4 q) { v = op(v, op(op(q.x, q.y), op(q.z, q.w))); }
  __device__ void merge(const AccExt &o) { v = op(v, o.v); }
  __device__ void shfl_merge(int off) { AccExt o; o.v = __shfl_down_sync(0xffffffffu, v, off); merge(o); }
  __device__ uint2 pack() const { return make_uint2(__builtin_bit_cast(uint32_t, v), 0u); }
  __device__ void unpack(uint2 q) { v = __builtin_bit_cast(T, q.x); }
};

// Product: int32 modulo 2^32 (exact), FP32 in FP32 arithmetic.
template <class T>
struct AccProd {
  static constexpr bool kIndexed = false;
  T v;
  __device__ static T mul(T a, T b) {
    if constexpr (std::is_same<T, float>::value) return __fmul_rn(a, b);
    else return (T)((uint32_t)a * (uint32_t)b);
  }
  __device__ void init() { v = T(1); }
  __device__ void add1(T x) { v = mul(v, x); }
  template <class V4>
  __device__ void add4(V4 q) { v = mul(v, mul(mul(q.x, q.y), mul(q.z, q.w))); }
  __device__ void merge(const AccProd &o) { v = mul(v, o.v); }
  __device__ void shfl_merge(int off) { AccProd o; o.v = __shfl_down_sync(0xffffffffu, v, off); merge(o); }
  __device__ uint2 pack() const { return make_uint2(__builtin_bit_cast(uint32_t, v), 0u); }
  __device__ void unpack(uint2 q) { v = __builtin_bit_cast(T, q.x); }
};

// Bitwise and / or / xor of int32 (OP 0 / 1 / 2).
template <int OP>
struct AccBits {
  static constexpr bool kIndexed = false;
  uint32_t v;
  __device__ static uint32_t op(uint32_t a, uint32_t b) { return OP == 0 ? (a & b) : OP == 1 ? (a | b) : (a ^ b); }
  __device__ void init() { v = OP == 0 ? 0xffffffffu : 0u; }
  __device__ void add1(int32_t x) { v = op(v, (uint32_t)x); }
  __device__ void add4(int4 q) { v = op(v, op(op((uint32_t)q.x, (uint32_t)q.y), op((uint32_t)q.z, (uint32_t)q.w))); }
  __device__ void merge(const AccBits &o) { v = op(v, o.v); }
  __device__ void shfl_merge(int off) { AccBits o; o.v = __shfl_down_sync(0xffffffffu, v, off); merge(o); }
  __device__ uint2 pack() const { return make_uint2(v, 0u); }
  __device__ void unpack(uint2 q) { v = q.x; }
};

// Arg-maximum / arg-minimum: the element index of the largest / smallest
// value, the smallest index among equal values; FP32 NaNs lose to every
// number (all NaN: the smallest index).  Index -1 is "no element" (the
// identity), which loses to every element.  The winner does not depend on
// the order of the merges.
template <class T, bool MAX>
__device__ __forceinline__ bool arg_better(T av, int32_t ai, T bv, int32_t bi) {
  if (bi < 0) return ai >= 0;
  if (ai < 0) return false;
  if constexpr (std::is_same<T, float>::value) {
    const bool an = av != av, bn = bv != bv;
    if (an != bn) return bn;
    if (an) return ai < bi;
  }
  if (av != bv) return MAX ? av > bv : av < bv;
  return ai < bi;
}
template <class T, bool MAX>
struct AccArg {
  static constexpr bool kIndexed = true;
  T v;
  int32_t i;
  __device__ void init() { v = T(0); i = -1; }
  __device__ void take(T x, int32_t j) {
    if (arg_better<T, MAX>(x, j, v, i)) { v = x; i = j; }
  }
  __device__ void add1_at(T x, int64_t j) { take(x, (int32_t)j); }
  template <class V4>
  __device__ void add4_at(V4 q, int64_t j) {
    take(q.x, (int32_t)j);
    take(q.y, (int32_t)(j + 1));
    take(q.z, (int32_t)(j + 2));
    take(q.w, (int32_t)(j + 3));
  }
  __device__ void merge(const AccArg &o) { take(o.v, o.i); }
  __device__ void shfl_merge(int off) {
    AccArg o;
    o.v = __shfl_down_sync(0xffffffffu, v, off);
    o.i = __shfl_down_sync(0xffffffffu, i, off);
    merge(o);
  }
  __device__ uint2 pack() const { return make_uint2(__builtin_bit_cast(uint32_t, v), (uint32_t)i); }
  __device__ void unpack(uint2 q) { v = __builtin_bit_cast(T, q.x); i = (int32_t)q.y; }
};

// Elements with their element index (used by the arg accumulators only).
template <class A, class T>
__device__ __forceinline__ void acc_add1(A &a, T x, int64_t idx) {
  if constexpr (A::kIndexed) a.add1_at(x, idx);
  else a.add1(x);
}
template <class A, class V4>
__device__ __forceinline__ void acc_add4(A &a, V4 q, int64_t idx) {
  if constexpr (A::kIndexed) a.add4_at(q, idx);
  else a.add4(q);
}

template <class A>
__device__ __forceinline__ void warp_merge(A &a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) a.shfl_merge(off);
}

// Block-wide merge; the result is valid in thread 0.  `sh` holds one A per warp.
template <class A, int THREADS>
__device__ __forceinline__ void block_merge(A &a, A *sh) {
  warp_merge(a);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = a;
  __syncthreads();
  if (w == 0) {
    if (lane < THREADS / 32) a = sh[lane];
    else a.init();
    warp_merge(a);
  }
}

// ---- affine maps evaluated element by element --------------------------
// Unsigned 32-bit division by a divisor fixed for the whole launch, by one
// multiply-high and shifts (Granlund and Montgomery, "Division by Invariant
// Integers using Multiplication", PLDI 1994, Figure 4.1): with
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0), t = mulhi(m, n),
// for every 32-bit n and 1 <= d <= 2^31.
struct FastDiv {
  uint32_t d, m, s1, s2;
};
inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while (l < 32 && (uint64_t(1) << l) < d) ++l;
  FastDiv f;
  f.d = d;
  f.m = (uint32_t)((((uint64_t(1) << l) - d) << 32) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 1 ? l - 1 : 0;
  return f;
}
__device__ __forceinline__ uint32_t fast_div(uint32_t n, const FastDiv &f) {
  const uint32_t t = __umulhi(f.m, n);
  return (t + ((n - t) >> f.s1)) >> f.s2;
}

// Drops extent-1 dims and merges neighbours that every stride set walks as
// one (outer stride = inner stride x inner extent), keeping the row-major
// logical order of the points.  ext/st[k] are arrays of nd entries; returns
// the new nd.
inline int canon_dims(int nd, int64_t *ext, int64_t *const *st, int nsets) {
  int m = 0;
  for (int i = 0; i < nd; ++i) {
    if (ext[i] == 1) continue;
    bool merge = m > 0;
    for (int k = 0; k < nsets && merge; ++k) merge = st[k][m - 1] == st[k][i] * ext[i];
    if (merge) {
      ext[m - 1] *= ext[i];
      for (int k = 0; k < nsets; ++k) st[k][m - 1] = st[k][i];
    } else {
      ext[m] = ext[i];
      for (int k = 0; k < nsets; ++k) st[k][m] = st[k][i];
      ++m;
    }
  }
  return m;
}

}  // namespace desc
