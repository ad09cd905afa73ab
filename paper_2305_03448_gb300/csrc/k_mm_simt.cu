// FP32 matrix multiplication on the CUDA cores (the non-tensor baseline).
//
// Classic register-tiled SGEMM: a CTA of 256 threads computes a 128 x 128
// tile of C; K advances in steps of 8 through double-buffered shared memory
// (A stored transposed so both operands are read as float4 rows).  Each
// thread accumulates an 8 x 8 block held as two 4 x 4 quadrants 64 apart,
// so the float4 shared-memory reads of a warp are bank-conflict-free.
// Global loads are register-prefetched one K step ahead.  Edges are guarded
// (zero fill on load, bounds on store).
#include "k_common.cuh"

namespace desc {
namespace {

constexpr int SBM = 128, SBN = 128, SBK = 8;

__global__ void __launch_bounds__(256) sgemm_kernel(const float *__restrict__ A, const float *__restrict__ B,
                                                    float *__restrict__ C, int64_t M, int64_t N, int64_t K,
                                                    int64_t lda, int64_t ldb, int64_t ldc) {
  __shared__ __align__(16) float As[2][SBK][SBM];
  __shared__ __align__(16) float Bs[2][SBK][SBN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t m0 = int64_t(blockIdx.y) * SBM, n0 = int64_t(blockIdx.x) * SBN;
  // loader coordinates: A tile 128 x 8 (thread: row tid/2, 4 k's), B tile 8 x 128 (row tid/32, 4 n's)
  const int a_r = tid / 2, a_k = (tid % 2) * 4;
  const int b_k = tid / 32, b_n = (tid % 32) * 4;
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
  auto load_b = [&](int64_t k0, float (&rb)[4]) {
    const int64_t k = k0 + b_k, n = n0 + b_n;
    if (b_vec && k < K && n + 4 <= N) {
      const float4 v = *reinterpret_cast<const float4 *>(B + k * ldb + n);
      rb[0] = v.x; rb[1] = v.y; rb[2] = v.z; rb[3] = v.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) rb[j] = (k < K && n + j < N) ? B[k * ldb + n + j] : 0.f;
    }
  };

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  float ra[4], rb[4];
  load_a(0, ra);
  load_b(0, rb);
#pragma unroll
  for (int j = 0; j < 4; ++j) As[0][a_k + j][a_r] = ra[j];
  *reinterpret_cast<float4 *>(&Bs[0][b_k][b_n]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
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
      const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][k][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][k][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      const int nb = buf ^ 1;
#pragma unroll
      for (int j = 0; j < 4; ++j) As[nb][a_k + j][a_r] = ra[j];
      *reinterpret_cast<float4 *>(&Bs[nb][b_k][b_n]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
      __syncthreads();
      buf = nb;
    }
  }
  const bool c_vec = (ldc % 4 == 0) && ((reinterpret_cast<uintptr_t>(C) & 15) == 0);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (r >= M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
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

int32_t launch_sgemm(const float *A, const float *B, float *C, int64_t M, int64_t N, int64_t K, int64_t lda,
                     int64_t ldb, int64_t ldc, desc_stream_t st) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  const int64_t gx = (N + SBN - 1) / SBN, gy = (M + SBM - 1) / SBM;
  if (gy > 65535 || gx >= (int64_t(1) << 31)) return DESC_ERR_UNSUPPORTED;
  sgemm_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, s>>>(A, B, C, M, N, K, lda, ldb, ldc);
  DESC_CUDA_TRY(cudaGetLastError());
  return DESC_OK;
}

}  // namespace desc
