// Copy through views: the tiled transpose and the general affine copy.
//
// Transpose: each CTA moves one TD x TD tile through a padded shared tile
// with 32 x 8 threads (the thread shape of the tiled transposes of Section 1;
// TD = 64 gives every thread 16 elements in flight), so that both the global
// reads (along input rows) and the global writes (along output rows) are
// coalesced 128-byte lines.  The padding of one word per row makes the
// column-wise shared-memory reads conflict-free.
//
// Affine copy: any pair of affine maps over a common domain; one element per
// thread and iteration, indices decoded from the domain extents.
#include <algorithm>

#include "k_bodies.cuh"
#include "k_common.cuh"

namespace desc {
namespace {

template <int TD, int BR>
__global__ void __launch_bounds__(32 * BR) transpose_kernel(const float *__restrict__ in,
                                                            float *__restrict__ out, int64_t R,
                                                            int64_t C, int64_t ld_in, int64_t ld_out,
                                                            int64_t bs_in, int64_t bs_out) {
  __shared__ float tile[TD][TD + 1];
  transpose_tile<TD, BR>(in, out, R, C, ld_in, ld_out, bs_in, bs_out, blockIdx.x, blockIdx.y, blockIdx.z,
                         threadIdx.x, threadIdx.y, tile);
}

struct CopyArgs {
  int32_t nd;
  int64_t extent[DESC_MAX_DIMS];
  int64_t istride[DESC_MAX_DIMS];
  int64_t ostride[DESC_MAX_DIMS];
  FastDiv div[DESC_MAX_DIMS];   // FAST: the extents as 32-bit invariant divisors
  int64_t ioff, ooff, total;
};

// One point per thread and step, decoded from its row-major logical index.
// FAST (fewer than 2^32 points, every extent <= 2^31): 32-bit decoding by
// multiply-high; otherwise 64-bit division.
template <bool FAST>
__global__ void __launch_bounds__(256) copy_affine_kernel(const uint32_t *__restrict__ in,
                                                          uint32_t *__restrict__ out,
                                                          const CopyArgs a) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < a.total; q += stride) {
    int64_t ie = a.ioff, oe = a.ooff;
    if (FAST) {
      uint32_t t = (uint32_t)q;
      for (int d = a.nd - 1; d > 0; --d) {
        const uint32_t qd = fast_div(t, a.div[d]);
        const int64_t c = int64_t(t - qd * a.div[d].d);
        ie += c * a.istride[d];
        oe += c * a.ostride[d];
        t = qd;
      }
      ie += int64_t(t) * a.istride[0];
      oe += int64_t(t) * a.ostride[0];
    } else {
      int64_t t = q;
      for (int d = a.nd - 1; d >= 0; --d) {
        const int64_t c = t % a.extent[d];
        t /= a.extent[d];
        ie += c * a.istride[d];
        oe += c * a.ostride[d];
      }
    }
    out[oe] = in[ie];
  }
}

}  // namespace

int transpose_candidates() { return kNumTransposeCands; }

int32_t launch_transpose(const float *in, float *out, int64_t R, int64_t C, int64_t ld_in,
                         int64_t ld_out, int64_t batch, int64_t bs_in, int64_t bs_out,
                         desc_stream_t st, int cand) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  if (R == 0 || C == 0 || batch == 0) return DESC_OK;
  constexpr int BR = 8;
  const int td = kTransposeTiles[(cand >= 0 && cand < kNumTransposeCands) ? cand : 0];
  if (td == 64 && R >= 64 && C >= 64) {   // 64 x 64 tiles: 16 loads in flight per thread
    constexpr int TD = 64;
    const int64_t gx = (C + TD - 1) / TD, gy = (R + TD - 1) / TD;
    if (gx >= (int64_t(1) << 31) || gy > 65535 || batch > 65535) return DESC_ERR_UNSUPPORTED;
    transpose_kernel<TD, BR><<<dim3((unsigned)gx, (unsigned)gy, (unsigned)batch), dim3(32, BR), 0, s>>>(
        in, out, R, C, ld_in, ld_out, bs_in, bs_out);
  } else {
    constexpr int TD = 32;
    const int64_t gx = (C + TD - 1) / TD, gy = (R + TD - 1) / TD;
    if (gx >= (int64_t(1) << 31) || gy > 65535 || batch > 65535) return DESC_ERR_UNSUPPORTED;
    transpose_kernel<TD, BR><<<dim3((unsigned)gx, (unsigned)gy, (unsigned)batch), dim3(32, BR), 0, s>>>(
        in, out, R, C, ld_in, ld_out, bs_in, bs_out);
  }
  DESC_CUDA_TRY(cudaGetLastError());
  return DESC_OK;
}

int32_t launch_copy_affine(const void *in, int64_t ioff, const int64_t *istride, void *out,
                           int64_t ooff, const int64_t *ostride, const int64_t *extent, int nd,
                           desc_stream_t st) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  CopyArgs a{};
  a.total = 1;
  for (int i = 0; i < nd; ++i) {
    a.extent[i] = extent[i];
    a.istride[i] = istride[i];
    a.ostride[i] = ostride[i];
    a.total *= extent[i];
  }
  a.ioff = ioff;
  a.ooff = ooff;
  if (a.total == 0) return DESC_OK;
  int64_t *sets[2] = {a.istride, a.ostride};
  a.nd = canon_dims(nd, a.extent, sets, 2);
  if (a.nd == 0) {                                     // a single point
    a.nd = 1;
    a.extent[0] = 1;
    a.istride[0] = a.ostride[0] = 0;
  }
  bool fast = a.total < (int64_t(1) << 32);
  for (int i = 0; i < a.nd; ++i) {
    fast = fast && a.extent[i] <= (int64_t(1) << 31);
    if (fast) a.div[i] = make_fastdiv((uint32_t)a.extent[i]);
  }
  const int64_t ctas = std::min<int64_t>((a.total + 255) / 256, 152 * 16);
  if (fast)
    copy_affine_kernel<true><<<(unsigned)ctas, 256, 0, s>>>(static_cast<const uint32_t *>(in),
                                                            static_cast<uint32_t *>(out), a);
  else
    copy_affine_kernel<false><<<(unsigned)ctas, 256, 0, s>>>(static_cast<const uint32_t *>(in),
                                                             static_cast<uint32_t *>(out), a);
  DESC_CUDA_TRY(cudaGetLastError());
  return DESC_OK;
}

}  // namespace desc
