// Copy through views: the tiled transpose and the general affine copy.
//
// Transpose: each CTA moves one TD x TD tile through a padded shared tile
// with 32 x 8 threads (the thread shape of the tiled transposes of Section 1;
// TD = 64 gives every thread 16 elements in flight), so that both the global
// reads (along input rows) and the global writes (along output rows) are
// coalesced 128-byte lines.  The padding of one word per row makes the
// column-wise shared-memory reads conflict-free.
//
// Affine copy: any pair of affine maps over a common domain.  Where the
// input map has a unit-stride dim and the output map another one, the copy
// is tiled over those two dims through shared memory (reads and writes both
// coalesced; the other dims are decoded once per CTA); otherwise one element
// per thread and iteration, indices decoded from the domain extents, with a
// unit-stride dim (if any) innermost so that at least one side coalesces.
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

// The tiled general copy: point (batch, r, c) of the domain reads
// in[ioff(batch) + r * ld_in + c] (c: the input's unit-stride dim) and writes
// out[ooff(batch) + c * ld_out + r] (r: the output's unit-stride dim).  Batch
// index z + blockIdx.z decoded over nb dims (extents / strides).
struct TiledCopyArgs {
  int32_t nb;
  int64_t R, C, ld_in, ld_out, batch;
  int64_t ext[DESC_MAX_DIMS], ist[DESC_MAX_DIMS], ost[DESC_MAX_DIMS];
  int64_t ioff, ooff;
};
// (8 CTAs of 256 threads per SM, as the hand-indexed transpose: 32 registers.)
__global__ void __launch_bounds__(256, 8) copy_tiled_kernel(const float *__restrict__ in, float *__restrict__ out,
                                                            const TiledCopyArgs a, int64_t z) {
  __shared__ float tile[64][65];
  int64_t io = a.ioff, oo = a.ooff, t = z + blockIdx.z;
  for (int d = a.nb - 1; d >= 0; --d) {
    const int64_t c = t % a.ext[d];
    t /= a.ext[d];
    io += c * a.ist[d];
    oo += c * a.ost[d];
  }
  transpose_tile<64, 8>(in + io, out + oo, a.R, a.C, a.ld_in, a.ld_out, 0, 0, blockIdx.x, blockIdx.y, 0,
                        threadIdx.x, threadIdx.y, tile);
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
  // unit-stride dims of the two maps (the longest, if several)
  int ua = -1, ub = -1;
  for (int i = 0; i < a.nd; ++i) {
    if (a.istride[i] == 1 && (ua < 0 || a.extent[i] > a.extent[ua])) ua = i;
    if (a.ostride[i] == 1 && (ub < 0 || a.extent[i] > a.extent[ub])) ub = i;
  }
  if (ua >= 0 && ub >= 0 && ua != ub && a.extent[ua] >= 16 && a.extent[ub] >= 16) {
    TiledCopyArgs t{};
    t.C = a.extent[ua];
    t.R = a.extent[ub];
    t.ld_in = a.istride[ub];
    t.ld_out = a.ostride[ua];
    t.batch = 1;
    for (int i = 0; i < a.nd; ++i) {
      if (i == ua || i == ub) continue;
      t.ext[t.nb] = a.extent[i];
      t.ist[t.nb] = a.istride[i];
      t.ost[t.nb] = a.ostride[i];
      t.batch *= a.extent[i];
      ++t.nb;
    }
    t.ioff = a.ioff;
    t.ooff = a.ooff;
    const int64_t gx = (t.C + 63) / 64, gy = (t.R + 63) / 64;
    if (gx < (int64_t(1) << 31) && gy <= 65535) {
      for (int64_t z = 0; z < t.batch; z += 65535) {   // launches of at most 65535 batch entries
        const unsigned gz = (unsigned)std::min<int64_t>(t.batch - z, 65535);
        copy_tiled_kernel<<<dim3((unsigned)gx, (unsigned)gy, gz), dim3(32, 8), 0, s>>>(
            static_cast<const float *>(in), static_cast<float *>(out), t, z);
      }
      DESC_CUDA_TRY(cudaGetLastError());
      return DESC_OK;
    }
  }
  // element-wise: a unit-stride dim innermost (the output's, else the input's)
  const int u = ub >= 0 ? ub : ua;
  if (u >= 0 && u != a.nd - 1) {
    std::swap(a.extent[u], a.extent[a.nd - 1]);
    std::swap(a.istride[u], a.istride[a.nd - 1]);
    std::swap(a.ostride[u], a.ostride[a.nd - 1]);
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
