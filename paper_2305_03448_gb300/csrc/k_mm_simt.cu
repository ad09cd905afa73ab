// FP32 matrix multiplication on the CUDA cores (the non-tensor baseline).
//
// Classic register-tiled SGEMM: a CTA of 256 threads computes a 128 x 128
// (or 128 x 256) tile of C; K advances in steps of 8 through double-buffered
// shared memory (A stored transposed so both operands are read as float4
// rows).  Each thread accumulates an 8 x 8 (or 8 x 16) block held as 4 x 4
// quadrants 64 rows / columns apart, so the float4 shared-memory reads of a
// warp are bank-conflict-free, and multiplies with the paired FP32 FMA
// (fma.rn.f32x2) on column pairs.
// Global loads are register-prefetched one K step ahead.  Edges are guarded
// (zero fill on load, bounds on store).
#include "k_common.cuh"

namespace desc {
namespace {

constexpr int SBM = 128, SBK = 8;

// NQ quadrants of 64 columns: a 128 x 64 NQ tile of C, each thread 8 x 4 NQ
// outputs (rows ty*4 .. and 64 + ty*4 .., columns q*64 + tx*4 ..).
template <int NQ>
__global__ void __launch_bounds__(256) sgemm_kernel(const float *__restrict__ A, const float *__restrict__ B,
                                                    float *__restrict__ C, int64_t M, int64_t N, int64_t K,
                                                    int64_t lda, int64_t ldb, int64_t ldc) {
  constexpr int SBN = 64 * NQ, VB = 2 * NQ;            // B columns per tile; B values each thread loads
  __shared__ __align__(16) float As[2][SBK][SBM];
  __shared__ __align__(16) float Bs[2][SBK][SBN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t m0 = int64_t(blockIdx.y) * SBM, n0 = int64_t(blockIdx.x) * SBN;
  // loader coordinates: A tile 128 x 8 (thread: row tid/2, 4 k's), B tile 8 x SBN (row tid/32, VB n's)
  const int a_r = tid / 2, a_k = (tid % 2) * 4;
  const int b_k = tid / 32, b_n = (tid % 32) * VB;
  const bool a_vec = (lda % 4 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
  const bool b_vec = (ldb % 4 == 0) && ((reinterpret_cast<uintptr_t>(B) & 15) == 0);

  auto load_a = [&](int64_t k0, float (&ra)[4]) {
    const int64_t r = m0 + a_r, k = k0 + a_k;
    if (a_vec && r < M && k + 4 <= K) {
      const float4 v = *reinterpret_cast<const float4 *>(A + r * lda + k);
      ra[0] = v.x; ra[1] = v.y; ra[2] = v.z; ra[3] = v.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) ra[j] = (r < M && k + j < K) ? A[r * lda + k + j] : 0.f;
    }
  };
  auto load_b = [&](int64_t k0, float (&rb)[VB]) {
    const int64_t k = k0 + b_k, n = n0 + b_n;
    if (b_vec && k < K && n + VB <= N) {
#pragma unroll
      for (int v4 = 0; v4 < VB / 4; ++v4) {
        const float4 v = *reinterpret_cast<const float4 *>(B + k * ldb + n + 4 * v4);
        rb[4 * v4] = v.x; rb[4 * v4 + 1] = v.y; rb[4 * v4 + 2] = v.z; rb[4 * v4 + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < VB; ++j) rb[j] = (k < K && n + j < N) ? B[k * ldb + n + j] : 0.f;
    }
  };

  // accumulators as column pairs (2p, 2p + 1): one fma.rn.f32x2 does the two
  // FMAs of a pair (per lane exactly fmaf), half the FMA instructions to issue
  unsigned long long acc2[8][2 * NQ];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int p = 0; p < 2 * NQ; ++p) acc2[i][p] = 0ull;

  float ra[4], rb[VB];
  auto store_b = [&](int nb) {
#pragma unroll
    for (int v4 = 0; v4 < VB / 4; ++v4)
      *reinterpret_cast<float4 *>(&Bs[nb][b_k][b_n + 4 * v4]) =
          make_float4(rb[4 * v4], rb[4 * v4 + 1], rb[4 * v4 + 2], rb[4 * v4 + 3]);
  };
  load_a(0, ra);
  load_b(0, rb);
#pragma unroll
  for (int j = 0; j < 4; ++j) As[0][a_k + j][a_r] = ra[j];
  store_b(0);
  __syncthreads();

  int buf = 0;
  for (int64_t k0 = 0; k0 < K; k0 += SBK) {
    const bool more = k0 + SBK < K;
    if (more) {
      load_a(k0 + SBK, ra);
      load_b(k0 + SBK, rb);
    }
#pragma unroll
    for (int k = 0; k < SBK; ++k) {
      const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][64 + ty * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      unsigned long long b2[2 * NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const float4 bq = *reinterpret_cast<const float4 *>(&Bs[buf][k][q * 64 + tx * 4]);
        asm("mov.b64 %0, {%1, %2};" : "=l"(b2[2 * q]) : "f"(bq.x), "f"(bq.y));
        asm("mov.b64 %0, {%1, %2};" : "=l"(b2[2 * q + 1]) : "f"(bq.z), "f"(bq.w));
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        unsigned long long a2;                          // a[i] in both halves
        asm("mov.b64 %0, {%1, %1};" : "=l"(a2) : "f"(a[i]));
#pragma unroll
        for (int p = 0; p < 2 * NQ; ++p)
          asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc2[i][p]) : "l"(a2), "l"(b2[p]));
      }
    }
    if (more) {
      const int nb = buf ^ 1;
#pragma unroll
      for (int j = 0; j < 4; ++j) As[nb][a_k + j][a_r] = ra[j];
      store_b(nb);
      __syncthreads();
      buf = nb;
    }
  }
  const bool c_vec = (ldc % 4 == 0) && ((reinterpret_cast<uintptr_t>(C) & 15) == 0);
  float acc[8][4 * NQ];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int p = 0; p < 2 * NQ; ++p)
      asm("mov.b64 {%0, %1}, %2;" : "=f"(acc[i][2 * p]), "=f"(acc[i][2 * p + 1]) : "l"(acc2[i][p]));
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (r >= M) continue;
#pragma unroll
    for (int h = 0; h < NQ; ++h) {
      const int64_t c = n0 + h * 64 + tx * 4;
      float *dst = C + r * ldc + c;
      if (c_vec && c + 4 <= N) {
        *reinterpret_cast<float4 *>(dst) =
            make_float4(acc[i][h * 4], acc[i][h * 4 + 1], acc[i][h * 4 + 2], acc[i][h * 4 + 3]);
      } else {
        for (int j = 0; j < 4; ++j)
          if (c + j < N) dst[j] = acc[i][h * 4 + j];
      }
    }
  }
}

}  // namespace

namespace {
template <int NQ>
int32_t launch_nq(const float *A, const float *B, float *C, int64_t M, int64_t N, int64_t K, int64_t lda,
                  int64_t ldb, int64_t ldc, cudaStream_t s) {
  const int64_t gx = (N + 64 * NQ - 1) / (64 * NQ), gy = (M + SBM - 1) / SBM;
  if (gy > 65535 || gx >= (int64_t(1) << 31)) return DESC_ERR_UNSUPPORTED;
  sgemm_kernel<NQ><<<dim3((unsigned)gx, (unsigned)gy), 256, 0, s>>>(A, B, C, M, N, K, lda, ldb, ldc);
  DESC_CUDA_TRY(cudaGetLastError());
  return DESC_OK;
}
}  // namespace

// 128 x 128 tiles (8 x 8 outputs per thread, 128 registers: two CTAs per
// SM).  With the paired FMAs it beats the 128 x 256 tile at every size
// measured on GB300 (8192^3: 19.6 against 20.8 ms; 4096^3: 2.59 against
// 3.02 ms); with single FMAs the wide tile had won at 8192^3 (22.7 against
// 23.6 ms).  All give the same bits.
int32_t launch_sgemm(const float *A, const float *B, float *C, int64_t M, int64_t N, int64_t K, int64_t lda,
                     int64_t ldb, int64_t ldc, desc_stream_t st) {
  return launch_nq<2>(A, B, C, M, N, K, lda, ldb, ldc, reinterpret_cast<cudaStream_t>(st));
}

}  // namespace desc
