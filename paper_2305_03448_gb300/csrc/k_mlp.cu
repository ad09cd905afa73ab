// The schedule cost model on the GPU: forward, backward, Adam and the
// candidate picker of a 3-layer MLP (F inputs, H hidden units twice, one
// output predicting log time).  FP32 throughout.
//
//   rows kernel   one warp per row: forward (each lane owns H/32 hidden
//                 units; activations are broadcast with shuffles), and for
//                 training the back-propagated deltas of that row
//   grad kernel   one thread per parameter, summing its row contributions in
//                 row order (deterministic, no atomics)
//   adam kernel   one thread per parameter
//   pick kernel   one warp per candidate, then the argmin (lowest index on ties)
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "k_common.cuh"

namespace desc {
namespace {

constexpr int kMaxF = 64, kMaxH = 64, kMaxCand = 8;

struct Layout {     // offsets of the parameter blocks
  int64_t W1, b1, W2, b2, w3, b3, total;
};
__host__ __device__ inline Layout layout(int F, int H) {
  Layout L;
  L.W1 = 0;
  L.b1 = L.W1 + int64_t(H) * F;
  L.W2 = L.b1 + H;
  L.b2 = L.W2 + int64_t(H) * H;
  L.w3 = L.b2 + H;
  L.b3 = L.w3 + H;
  L.total = L.b3 + 1;
  return L;
}

// Per-row scratch: h1, h2, dz1, dz2 (H each), dy, squared error.
__host__ __device__ inline int64_t row_stride(int H) { return 4 * int64_t(H) + 2; }

// Forward of one row by one warp.  Lane l owns hidden units l and l + 32.
// Returns y (in every lane); z1/z2/h1/h2 of the owned units in the arrays.
__device__ __forceinline__ float forward_row(const float *__restrict__ P, int F, int H, const float *__restrict__ x,
                                             float (&z1)[kMaxH / 32], float (&z2)[kMaxH / 32], float (&h1)[kMaxH / 32],
                                             float (&h2)[kMaxH / 32]) {
  const Layout L = layout(F, H);
  const int lane = threadIdx.x & 31, per = H / 32;
  for (int u = 0; u < per; ++u) {
    const int j = lane + 32 * u;
    float acc = P[L.b1 + j];
    for (int f = 0; f < F; ++f) acc = fmaf(P[L.W1 + int64_t(j) * F + f], x[f], acc);
    z1[u] = acc;
    h1[u] = fmaxf(acc, 0.f);
  }
  for (int u = 0; u < per; ++u) {
    const int j = lane + 32 * u;
    float acc = P[L.b2 + j];
    for (int i = 0; i < H; ++i) {
      const float hi = __shfl_sync(0xffffffffu, (i >> 5) == 0 ? h1[0] : h1[1], i & 31);
      acc = fmaf(P[L.W2 + int64_t(j) * H + i], hi, acc);
    }
    z2[u] = acc;
    h2[u] = fmaxf(acc, 0.f);
  }
  float y = 0.f;
  for (int u = 0; u < per; ++u) y = fmaf(P[L.w3 + lane + 32 * u], h2[u], y);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) y += __shfl_xor_sync(0xffffffffu, y, off);
  return y + P[L.b3];
}

template <bool TRAIN>
__global__ void __launch_bounds__(256) mlp_rows_kernel(const float *__restrict__ P, int F, int H,
                                                       const float *__restrict__ X, const float *__restrict__ t,
                                                       int64_t rows, float *__restrict__ y_out,
                                                       float *__restrict__ scratch) {
  const int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (r >= rows) return;
  const int lane = threadIdx.x & 31, per = H / 32;
  const float *x = X + r * F;
  float z1[kMaxH / 32], z2[kMaxH / 32], h1[kMaxH / 32], h2[kMaxH / 32];
  const float y = forward_row(P, F, H, x, z1, z2, h1, h2);
  if (y_out && lane == 0) y_out[r] = y;
  if (!TRAIN) return;
  const Layout L = layout(F, H);
  float *S = scratch + r * row_stride(H);
  const float err = y - t[r];
  const float dy = 2.f * err / float(rows);
  float dz2[kMaxH / 32], dz1[kMaxH / 32];
  for (int u = 0; u < per; ++u) dz2[u] = z2[u] > 0.f ? dy * P[L.w3 + lane + 32 * u] : 0.f;
  for (int u = 0; u < per; ++u) {
    const int i = lane + 32 * u;
    float acc = 0.f;
    for (int j = 0; j < H; ++j) {
      const float dj = __shfl_sync(0xffffffffu, (j >> 5) == 0 ? dz2[0] : dz2[1], j & 31);
      acc = fmaf(P[L.W2 + int64_t(j) * H + i], dj, acc);
    }
    dz1[u] = z1[u] > 0.f ? acc : 0.f;
  }
  for (int u = 0; u < per; ++u) {
    const int j = lane + 32 * u;
    S[j] = h1[u];
    S[H + j] = h2[u];
    S[2 * H + j] = dz1[u];
    S[3 * H + j] = dz2[u];
  }
  if (lane == 0) {
    S[4 * H] = dy;
    S[4 * H + 1] = err * err;
  }
}

__global__ void __launch_bounds__(256) mlp_grad_kernel(int F, int H, const float *__restrict__ X, int64_t rows,
                                                       const float *__restrict__ scratch, float *__restrict__ grad) {
  const Layout L = layout(F, H);
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= L.total) return;
  const int64_t rs = row_stride(H);
  float acc = 0.f;
  if (p < L.b1) {                                  // W1[j][f]: dz1[j] x[f]
    const int j = int(p / F), f = int(p % F);
    for (int64_t r = 0; r < rows; ++r) acc = fmaf(scratch[r * rs + 2 * H + j], X[r * F + f], acc);
  } else if (p < L.W2) {                           // b1[j]: dz1[j]
    const int j = int(p - L.b1);
    for (int64_t r = 0; r < rows; ++r) acc += scratch[r * rs + 2 * H + j];
  } else if (p < L.b2) {                           // W2[j][i]: dz2[j] h1[i]
    const int j = int((p - L.W2) / H), i = int((p - L.W2) % H);
    for (int64_t r = 0; r < rows; ++r) acc = fmaf(scratch[r * rs + 3 * H + j], scratch[r * rs + i], acc);
  } else if (p < L.w3) {                           // b2[j]: dz2[j]
    const int j = int(p - L.b2);
    for (int64_t r = 0; r < rows; ++r) acc += scratch[r * rs + 3 * H + j];
  } else if (p < L.b3) {                           // w3[j]: dy h2[j]
    const int j = int(p - L.w3);
    for (int64_t r = 0; r < rows; ++r) acc = fmaf(scratch[r * rs + 4 * H], scratch[r * rs + H + j], acc);
  } else {                                         // b3: dy
    for (int64_t r = 0; r < rows; ++r) acc += scratch[r * rs + 4 * H];
  }
  grad[p] = acc;
}

__global__ void __launch_bounds__(256) mlp_adam_kernel(float *__restrict__ P, const float *__restrict__ g,
                                                       float *__restrict__ m, float *__restrict__ v, int64_t n,
                                                       float lr, float b1, float b2, float eps, float c1, float c2) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void __launch_bounds__(kMaxCand * 32) mlp_pick_kernel(const float *__restrict__ P, int F, int H,
                                                                 const float *__restrict__ Xc, int ncand,
                                                                 float *__restrict__ pred, int *__restrict__ best) {
  __shared__ float sp[kMaxCand];
  const int w = threadIdx.x >> 5;
  if (w < ncand) {
    float z1[kMaxH / 32], z2[kMaxH / 32], h1[kMaxH / 32], h2[kMaxH / 32];
    const float y = forward_row(P, F, H, Xc + int64_t(w) * F, z1, z2, h1, h2);
    if ((threadIdx.x & 31) == 0) sp[w] = y;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int b = 0;
    for (int c = 1; c < ncand; ++c)
      if (sp[c] < sp[b]) b = c;
    *best = b;
    for (int c = 0; c < ncand; ++c) pred[c] = sp[c];
  }
}

// Staging for desc_tune_predict: the candidates' features and the pick.  One
// copy per device, shared by every caller, so each prediction holds g_pick_mu
// from the copy in to the copy out.
__device__ float g_pick_x[kMaxCand * kMaxF];
__device__ float g_pick_pred[kMaxCand];
__device__ int g_pick_best;
std::mutex g_pick_mu;

bool shape_ok(int F, int H) { return F >= 1 && F <= kMaxF && (H == 32 || H == 64); }

}  // namespace

int32_t mlp_pick_device(const float *params, int32_t F, int32_t H, const float *Xhost, int32_t ncand,
                        desc_stream_t st, int32_t *best) {
  if (!shape_ok(F, H) || ncand < 1 || ncand > kMaxCand) return DESC_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  std::lock_guard<std::mutex> lock(g_pick_mu);
  DESC_CUDA_TRY(cudaMemcpyToSymbolAsync(g_pick_x, Xhost, size_t(ncand) * F * sizeof(float), 0,
                                        cudaMemcpyHostToDevice, s));
  float *px;
  float *pp;
  int *pb;
  DESC_CUDA_TRY(cudaGetSymbolAddress(reinterpret_cast<void **>(&px), g_pick_x));
  DESC_CUDA_TRY(cudaGetSymbolAddress(reinterpret_cast<void **>(&pp), g_pick_pred));
  DESC_CUDA_TRY(cudaGetSymbolAddress(reinterpret_cast<void **>(&pb), g_pick_best));
  mlp_pick_kernel<<<1, kMaxCand * 32, 0, s>>>(params, F, H, px, ncand, pp, pb);
  DESC_CUDA_TRY(cudaGetLastError());
  int b = 0;
  DESC_CUDA_TRY(cudaMemcpyFromSymbolAsync(&b, g_pick_best, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  DESC_CUDA_TRY(cudaStreamSynchronize(s));
  *best = b;
  return DESC_OK;
}

}  // namespace desc

using namespace desc;

extern "C" int32_t desc_mlp_param_count(int32_t F, int32_t H, int64_t *count) {
  if (!count || !shape_ok(F, H)) return DESC_ERR_INVALID_ARG;
  *count = layout(F, H).total;
  return DESC_OK;
}

extern "C" int32_t desc_mlp_workspace_size(int32_t F, int32_t H, int64_t rows, size_t *bytes) {
  if (!bytes || !shape_ok(F, H) || rows < 0) return DESC_ERR_INVALID_ARG;
  *bytes = size_t(rows) * row_stride(H) * sizeof(float);
  return DESC_OK;
}

extern "C" int32_t desc_mlp_forward(const float *params, int32_t F, int32_t H, const float *X, int64_t rows,
                                    float *y, void *ws, size_t ws_bytes, desc_stream_t st) {
  (void)ws;
  (void)ws_bytes;
  if (!shape_ok(F, H) || rows < 0 || !params || (rows && (!X || !y))) return DESC_ERR_INVALID_ARG;
  if (!rows) return DESC_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  const int64_t ctas = (rows * 32 + 255) / 256;
  mlp_rows_kernel<false><<<(unsigned)ctas, 256, 0, s>>>(params, F, H, X, nullptr, rows, y, nullptr);
  DESC_CUDA_TRY(cudaGetLastError());
  return DESC_OK;
}

extern "C" int32_t desc_mlp_backward(const float *params, int32_t F, int32_t H, const float *X, const float *t,
                                     int64_t rows, float *grad, void *ws, size_t ws_bytes, desc_stream_t st) {
  if (!shape_ok(F, H) || rows < 1 || !params || !X || !t || !grad) return DESC_ERR_INVALID_ARG;
  if (!ws || ws_bytes < size_t(rows) * row_stride(H) * sizeof(float)) return DESC_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  float *scratch = static_cast<float *>(ws);
  mlp_rows_kernel<true><<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(params, F, H, X, t, rows, nullptr,
                                                                           scratch);
  const int64_t P = layout(F, H).total;
  mlp_grad_kernel<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(F, H, X, rows, scratch, grad);
  DESC_CUDA_TRY(cudaGetLastError());
  return DESC_OK;
}

extern "C" int32_t desc_mlp_adam(float *params, const float *grad, float *m, float *v, int64_t count, int32_t step,
                                 float lr, float beta1, float beta2, float eps, desc_stream_t st) {
  if (!params || !grad || !m || !v || count < 0 || step < 1) return DESC_ERR_INVALID_ARG;
  if (!count) return DESC_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  const float c1 = float(1.0 - std::pow(double(beta1), step)), c2 = float(1.0 - std::pow(double(beta2), step));
  mlp_adam_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(params, grad, m, v, count, lr, beta1, beta2, eps,
                                                                 c1, c2);
  DESC_CUDA_TRY(cudaGetLastError());
  return DESC_OK;
}

extern "C" int32_t desc_mlp_train(float *params, float *grad, float *m, float *v, int32_t F, int32_t H,
                                  const float *X, const float *t, int64_t rows, int32_t epochs, int32_t batch,
                                  float lr, void *ws, size_t ws_bytes, desc_stream_t st, float *loss) {
  if (!shape_ok(F, H) || rows < 1 || epochs < 1 || batch < 1) return DESC_ERR_INVALID_ARG;
  if (!ws || ws_bytes < size_t(rows) * row_stride(H) * sizeof(float)) return DESC_ERR_WORKSPACE;
  const int64_t P = layout(F, H).total;
  int32_t step = 0, r;
  for (int e = 0; e < epochs; ++e)
    for (int64_t b0 = 0; b0 < rows; b0 += batch) {
      const int64_t B = std::min<int64_t>(batch, rows - b0);
      if ((r = desc_mlp_backward(params, F, H, X + b0 * F, t + b0, B, grad, ws, ws_bytes, st)) != DESC_OK) return r;
      if ((r = desc_mlp_adam(params, grad, m, v, P, ++step, lr, 0.9f, 0.999f, 1e-8f, st)) != DESC_OK) return r;
    }
  if (loss) {   // mean squared error of the final parameters over all rows
    cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
    float *scratch = static_cast<float *>(ws);
    mlp_rows_kernel<true><<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(params, F, H, X, t, rows, nullptr,
                                                                             scratch);
    DESC_CUDA_TRY(cudaGetLastError());
    std::vector<float> sq(size_t(rows) * row_stride(H));
    DESC_CUDA_TRY(cudaMemcpyAsync(sq.data(), scratch, sq.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
    DESC_CUDA_TRY(cudaStreamSynchronize(s));
    double acc = 0;
    for (int64_t i = 0; i < rows; ++i) acc += sq[size_t(i * row_stride(H) + 4 * H + 1)];
    *loss = float(acc / double(rows));
  }
  return DESC_OK;
}

extern "C" int32_t desc_mlp_pick(const float *params, int32_t F, int32_t H, const float *Xcand, int32_t ncand,
                                 float *pred, int32_t *best, desc_stream_t st) {
  if (!shape_ok(F, H) || ncand < 1 || ncand > kMaxCand || !params || !Xcand || !pred || !best)
    return DESC_ERR_INVALID_ARG;
  mlp_pick_kernel<<<1, kMaxCand * 32, 0, reinterpret_cast<cudaStream_t>(st)>>>(params, F, H, Xcand, ncand, pred,
                                                                             best);
  DESC_CUDA_TRY(cudaGetLastError());
  return DESC_OK;
}
