// Schedule candidates of every tunable op, in one place: the kernels launch
// from these tables and the cost model's features describe the same entries,
// so the two cannot drift apart.  Candidate 0 is each op's default.
#pragma once

#include <cstdint>

namespace desc {

// Chunked reduce: vectors of four elements in flight per thread, the CTA
// count the chunking aims at (1216 = 8 CTAs on each of 152 SMs) and the load
// path (0: evict-first streaming loads, 1: read-only path without L1
// allocation).
struct ReduceCand {
  int unroll;
  int64_t target_ctas;
  int nc;
};
constexpr ReduceCand kReduceCands[] = {{8, 1216, 0}, {4, 1216, 0}, {8, 608, 0}, {4, 2432, 0},
                                       {8, 2432, 0}, {8, 304, 0},  {4, 2432, 1}, {8, 1216, 1}};
constexpr int kNumReduceCands = sizeof(kReduceCands) / sizeof(kReduceCands[0]);

// Look-back scans (plain, per-level segments and CSR segments): sub-tiles of
// 4096 elements per tile.
constexpr int kScanSubTile = 4096;
constexpr int kScanSubCands[] = {4, 2, 1};
constexpr int kNumScanCands = sizeof(kScanSubCands) / sizeof(kScanSubCands[0]);

// Segmented (CSR) scans: the look-back scan over tiles of 4096 x sub points
// (threads = 0: every segment shares the tiles), or one group of `threads`
// threads per segment, walking it in steps of threads x 4 points.
struct SegCand {
  int sub;
  int threads;
};
constexpr SegCand kSegCands[] = {{4, 0}, {2, 0}, {1, 0}, {0, 32}, {0, 256}};
constexpr int kNumSegCands = sizeof(kSegCands) / sizeof(kSegCands[0]);

// Tiled transpose: square tiles of this many rows and columns.
constexpr int kTransposeTiles[] = {64, 32};
constexpr int kNumTransposeCands = sizeof(kTransposeTiles) / sizeof(kTransposeTiles[0]);

// Tensor-core matmul: CTA pairs (cta_group::2 over 256-row tiles, where the
// 128-row tiles pair up) or single CTAs over 128-row tiles; the
// rasterisation group in 128-row tile rows; the pair tile's width in units of
// 256 columns.
struct MmCand {
  int pairs;
  int group_rows;
  int width;
};
constexpr MmCand kMmCands[] = {{1, 16, 1}, {0, 16, 1}, {1, 4, 1}, {0, 4, 1}, {1, 16, 2}, {1, 4, 2}};
constexpr int kNumMmCands = sizeof(kMmCands) / sizeof(kMmCands[0]);

}  // namespace desc
