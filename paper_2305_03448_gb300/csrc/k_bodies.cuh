// Block bodies shared by more than one kernel: the work of one CTA, with its
// block coordinates passed in, so that a kernel can run it for a part of its
// grid (the split launches) as well as for the whole grid.
#pragma once

#include <cstdint>

namespace desc {

// One TD x TD tile of out = in^T (row-major R x C -> C x R, batch bz) through
// a padded shared tile, 32 x BR threads (tx, ty): reads along input rows and
// writes along output rows are coalesced 128-byte lines, and the padding of
// one word per row keeps the column-wise shared reads conflict-free.
template <int TD, int BR>
__device__ __forceinline__ void transpose_tile(const float *__restrict__ in, float *__restrict__ out, int64_t R,
                                               int64_t C, int64_t ld_in, int64_t ld_out, int64_t bs_in,
                                               int64_t bs_out, int64_t bx, int64_t by, int64_t bz, int tx, int ty,
                                               float (&tile)[TD][TD + 1]) {
  const float *src = in + bz * bs_in;
  float *dst = out + bz * bs_out;
  const int64_t r0 = by * TD, c0 = bx * TD;
  const bool interior = (r0 + TD <= R) && (c0 + TD <= C);
  if (interior) {
#pragma unroll
    for (int j = 0; j < TD; j += BR)
#pragma unroll
      for (int i = 0; i < TD; i += 32)
        tile[ty + j][tx + i] = __ldcs(src + (r0 + ty + j) * ld_in + c0 + tx + i);
  } else {
    for (int j = 0; j < TD; j += BR)
      for (int i = 0; i < TD; i += 32) {
        const int64_t r = r0 + ty + j, c = c0 + tx + i;
        if (r < R && c < C) tile[ty + j][tx + i] = src[r * ld_in + c];
      }
  }
  __syncthreads();
  // out[c][r] = in[r][c]: output row c0 + ty + j, output column r0 + tx + i
  if (interior) {
#pragma unroll
    for (int j = 0; j < TD; j += BR)
#pragma unroll
      for (int i = 0; i < TD; i += 32)
        __stcs(dst + (c0 + ty + j) * ld_out + r0 + tx + i, tile[tx + i][ty + j]);
  } else {
    for (int j = 0; j < TD; j += BR)
      for (int i = 0; i < TD; i += 32) {
        const int64_t c = c0 + ty + j, r = r0 + tx + i;
        if (r < R && c < C) dst[c * ld_out + r] = tile[tx + i][ty + j];
      }
  }
}

}  // namespace desc
