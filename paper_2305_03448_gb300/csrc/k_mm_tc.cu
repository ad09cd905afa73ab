// Tensor-core matrix multiplication on sm_103a: tcgen05.mma with the
// accumulator in tensor memory (TMEM), operands staged by TMA.
//
// C (M x N, FP32) = sum over the products (i, j) of A_i B_j, where A_i and
// B_j are BF16 planes written by the split pass: A_i is M x K (K-major) and
// B_j is stored transposed, N x K (K-major).  Plain BF16 has one product;
// the 3-term split has six (i + j <= 2).  All products accumulate into one
// FP32 accumulator in TMEM.
//
// Accuracy: every product's K range is split in two halves whose sums are
// added in FP32 by the epilogue, so no sum takes more than half of the
// K' = products x K terms: two TMEM accumulators (all 512 columns) for
// 256-column tiles, or two phases of one 512-column accumulator set for
// 512-column tiles (the first half's sums parked in workspace) -- the same
// sums in the same order, bit-identical results.
// Stage order: product by product, each over all of K.  (Taking all products
// of a K block in turn would re-read planes while still in L2, but it mixes
// the small correction products into the running sum earlier and measured
// 1.6x the accumulation error of this order.)
//
// One CTA computes a 128 x 256 tile of C (192 threads, 1 CTA per SM):
//   warp 0, one lane   TMA producer: A and B K-blocks of 64 into a 4-stage
//                      ring (128-byte swizzle), one mbarrier per stage
//   warp 1, one lane   MMA issuer: 4 x tcgen05.mma (M128 N256 K16) per stage,
//                      tcgen05.commit frees the stage; warp 1 also owns the
//                      TMEM allocation (512 columns)
//   warps 2..5         epilogue: tcgen05.ld 32 rows x 32 columns per warp and
//                      step (warp w reads TMEM lanes 32 (w mod 4) ...), FP32 stores
//                      through TMA from a staging buffer
// Pairs (mm_tc_pair_kernel<NW>, used when the 128-row tiles pair up): the two
// CTAs of a thread-block cluster compute one 256 x 256 NW tile with NW
// tcgen05.mma.cta_group::2 (M256 N256 K16) per K step.  Each CTA stages its
// own 128 rows of A and its own 128 of each 256 B rows, so for NW = 1 a
// stage is 32 KB instead of 48 KB for the same work per SM (six stages), and
// for NW = 2 48 KB for twice the work (four stages): the operand stream into
// each SM, not the tensor pipe, had set the pace of the 256 x 256 tiles.
// The even CTA issues the MMAs for both; its full barriers count the bytes
// of both CTAs' copies, its MMA commits free the stages and publish the
// accumulators in both CTAs, and the epilogue warps of both CTAs (each reads
// its own 128 accumulator rows) report to it.
// Every wait is bounded: a waiter that gives up sets an abort flag in shared
// memory and records DESC_ERR_DEVICE_TIMEOUT; the producer then waits, again
// with a limit, for the copies it has in flight, and TMEM is always freed.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "k_common.cuh"

namespace desc {

__device__ int g_mm_status;

namespace {

constexpr int BM = 128, BN = 256, BK = 64, UK = 16;
constexpr int kStages = 4;
constexpr int kABytes = BM * BK * 2;             // 16 KB
constexpr int kBBytes = BN * BK * 2;             // 32 KB
constexpr int kStageBytes = kABytes + kBBytes;
constexpr int kTmemCols = 512;                  // two 256-column accumulators
constexpr int kMmThreads = 192;
// Epilogue staging for the TMA stores of C: per epilogue warp two buffers of
// 32 rows x 32 FP32 (128-byte swizzle), after the operand stages.
constexpr int kEpiBufBytes = 32 * 32 * 4;
constexpr int kEpiBytes = 4 * 2 * kEpiBufBytes;
constexpr int kSmemBytes = kStages * kStageBytes + kEpiBytes + 1024 + 256;
constexpr long long kWaitBudget = 1ll << 32;     // clock cycles, about two seconds
constexpr int kGroupM = 16;                      // tile rows per rasterisation group

struct Products {
  int n;
  int pa[8];
  int pb[8];
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity.  false: gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > kWaitBudget) {
      *abort = 1;
      atomicCAS(&g_mm_status, 0, (int)DESC_ERR_DEVICE_TIMEOUT);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *tm, uint64_t *bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
      ::"r"(smem_u32(dst)), "l"(tm), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows
// of 64 BF16 (128 B), 8-row core groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);     // start address
  d |= (uint64_t)1 << 16;                               // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;                     // stride byte offset
  d |= (uint64_t)1 << 46;                               // descriptor version
  d |= (uint64_t)2 << 61;                               // 128-byte swizzle
  return d;
}
// Instruction descriptor (kind::f16): FP32 accumulator, BF16 A and B, both
// K-major, N = BN, M = BM.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 32 consecutive outputs of one row of C (columns col .. col + 31).
__device__ __forceinline__ void store_row32(float *__restrict__ C, int64_t row, int64_t col, int64_t M, int64_t N,
                                            int64_t ldc, bool vec, const uint32_t (&r)[32]) {
  if (row >= M) return;
  float *dst = C + row * ldc + col;
  if (vec && col + 32 <= N) {
#pragma unroll
    for (int j = 0; j < 32; j += 4)
      __stcs(reinterpret_cast<float4 *>(dst + j), make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                                             __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3])));
  } else {
    for (int j = 0; j < 32; ++j)
      if (col + j < N) dst[j] = __uint_as_float(r[j]);
  }
}

// ---- epilogue stores of C through TMA ------------------------------------
// A warp holds 32 rows of C (one per lane) x 32 columns per step.  Writing
// them row by row from registers makes every warp store touch 32 lines; here
// each lane puts its row into a 128-byte-swizzled staging buffer (16-byte
// chunk k of row r at chunk k ^ (r mod 8): conflict-free) and one lane
// stores the 32 x 32 box with cp.async.bulk.tensor, which clips at the edges
// of C.  Two buffers per warp: a buffer is rewritten only after the store
// issued from it two steps earlier has read it.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *tm, const void *src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(tm),
               "r"(smem_u32(src)), "r"(x), "r"(y)
               : "memory");
}
struct EpiStage {
  unsigned char *buf;   // this warp's two buffers (1024-byte aligned)
  int n;                // boxes issued so far
};
__device__ __forceinline__ void epi_store_box(EpiStage &e, const CUtensorMap *tm, int x, int y, bool inside,
                                              int lane, const uint32_t (&r)[32]) {
  unsigned char *b = e.buf + (e.n & 1) * kEpiBufBytes;
  if (e.n >= 2) {
    if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
    __syncwarp();
  }
#pragma unroll
  for (int k = 0; k < 8; ++k)
    *reinterpret_cast<uint4 *>(b + lane * 128 + ((k ^ (lane & 7)) << 4)) =
        make_uint4(r[4 * k], r[4 * k + 1], r[4 * k + 2], r[4 * k + 3]);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if (lane == 0) {                                   // one group per box, empty where it lies outside C
    if (inside) tma_store_2d(tm, b, x, y);
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  }
  ++e.n;
}
// Every store of this lane complete (before the CTA leaves).
__device__ __forceinline__ void epi_drain(int lane) {
  if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  __syncwarp();
}

// Tile order: groups of kGroupM tile rows, column by column inside a group,
// so that the operand panels a wave of CTAs touches stay in L2.
struct TileMap {
  int Mt, Nt, group_m;
};
__device__ __forceinline__ void tile_coords(int t, const TileMap &g, int &mt, int &nt) {
  const int per_group = g.group_m * g.Nt;
  const int first = (t / per_group) * g.group_m;
  const int gm = min(g.Mt - first, g.group_m);
  const int r = t % per_group;
  mt = first + r % gm;
  nt = r / gm;
}

// Persistent: CTA b takes tiles b, b + gridDim.x, ...  The producer streams
// the operand stages of consecutive tiles without a break, so the next tile's
// loads overlap the current tile's epilogue.  Accumulator sets in TMEM:
// with one product (BF16) two sets of 256 columns alternate between tiles,
// so the epilogue of tile i overlaps the MMAs of tile i + 1; with the split
// forms one set spans both 256-column accumulators (the two K halves).
__global__ void __launch_bounds__(kMmThreads, 1)
    mm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const __grid_constant__ CUtensorMap tmC, float *__restrict__ C, int64_t M, int64_t N, int64_t ldc,
                 int kblocks, Products prods, TileMap tm, int ntiles, int split_acc, int tma_c) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                          ~uintptr_t(1023));
  unsigned char *sA = smem;
  unsigned char *sB = smem + kStages * kABytes;
  unsigned char *sEpi = smem + kStages * kStageBytes;
  uint64_t *full = reinterpret_cast<uint64_t *>(sEpi + kEpiBytes);
  uint64_t *empty = full + kStages;
  uint64_t *tfull = empty + kStages;
  uint64_t *tempty = tfull + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tempty + 2);
  volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 4);                        // one arrival per epilogue warp
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int per_tile = kblocks * prods.n;              // stages per tile
  const int nsets = split_acc ? 1 : 2;

  if (warp == 0) {
    if (lane == 0) {                                   // ---- TMA producer
      int it = 0, issued = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int mt, nt;
        tile_coords(t, tm, mt, nt);
        for (int j = 0; j < per_tile; ++j, ++it) {
          const int s = it % kStages;
          const uint32_t ph = (it / kStages) & 1;
          if (!mbar_wait(&empty[s], ph ^ 1, abort)) { ok = false; break; }
          const int p = j / kblocks, kb = j % kblocks;
          mbar_expect_tx(&full[s], kStageBytes);
          tma_load_3d(sA + s * kABytes, &tmA, &full[s], kb * BK, mt * BM, prods.pa[p]);
          tma_load_3d(sB + s * kBBytes, &tmB, &full[s], kb * BK, nt * BN, prods.pb[p]);
          issued = it + 1;
        }
      }
      if (*abort) {                                    // copies still in flight: wait, bounded
        for (int i = std::max(0, issued - kStages); i < issued; ++i) {
          const long long t0 = clock64();
          while (!mbar_try_wait(&full[i % kStages], (i / kStages) & 1) && clock64() - t0 < kWaitBudget) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {                                   // ---- MMA issuer
      const int half = kblocks / 2;
      int it = 0, li = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++li) {
        const int si = li % nsets;
        const uint32_t use = (uint32_t)(li / nsets);
        if (!mbar_wait(&tempty[si], (use & 1) ^ 1, abort)) break;   // epilogue has drained this set
        tc_fence_after();
        for (int j = 0; j < per_tile; ++j, ++it) {
          const int s = it % kStages;
          const uint32_t ph = (it / kStages) & 1;
          if (!mbar_wait(&full[s], ph, abort)) { ok = false; break; }
          tc_fence_after();
          const int p = j / kblocks, kb = j % kblocks;
          int acc;
          bool first;
          if (split_acc) {                             // K halves in two accumulators
            acc = (half > 0 && kb >= half) ? 1 : 0;
            first = p == 0 && kb == (acc ? half : 0);
          } else {
            acc = si;
            first = j == 0;
          }
          const uint32_t d = tmem + (uint32_t)(acc * BN);
          const uint32_t a0 = smem_u32(sA + s * kABytes), b0 = smem_u32(sB + s * kBBytes);
#pragma unroll
          for (int k = 0; k < BK / UK; ++k)
            umma_bf16(d, sdesc(a0 + k * UK * 2), sdesc(b0 + k * UK * 2), (first && k == 0) ? 0u : 1u);
          umma_commit(&empty[s]);                      // stage reusable once these MMAs finish
        }
        if (ok) umma_commit(&tfull[si]);               // this tile's accumulators complete
      }
    }
  } else {                                             // ---- epilogue, warps 2..5
    const int q = warp & 3;                            // TMEM lanes 32 q .. 32 q + 31
    const bool vec = ((ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(C) & 15) == 0);
    const bool two = split_acc && kblocks / 2 > 0;
    EpiStage es{sEpi + q * 2 * kEpiBufBytes, 0};
    int li = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++li) {
      const int si = li % nsets;
      const uint32_t use = (uint32_t)(li / nsets);
      if (!mbar_wait(&tfull[si], use & 1, abort)) break;
      tc_fence_after();
      int mt, nt;
      tile_coords(t, tm, mt, nt);
      const int64_t row = int64_t(mt) * BM + q * 32 + lane;
      const int64_t n0 = int64_t(nt) * BN;
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(split_acc ? 0 : si * BN);
#pragma unroll 1
      for (int c = 0; c < BN / 32; ++c) {
        uint32_t r[32];
        tmem_ld32(base + (uint32_t)(c * 32), r);
        if (two) {
          uint32_t r1[32];
          tmem_ld32(base + (uint32_t)(BN + c * 32), r1);
#pragma unroll
          for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(__fadd_rn(__uint_as_float(r[j]), __uint_as_float(r1[j])));
        }
        const int64_t col = n0 + c * 32, row0 = row - lane;
        if (tma_c)
          epi_store_box(es, &tmC, (int)col, (int)row0, row0 < M && col < N, lane, r);
        else
          store_row32(C, row, col, M, N, ldc, vec, r);
      }
      tc_fence_before();                               // TMEM reads done before the set is reused
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[si]);
    }
    epi_drain(lane);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

// ---- pairs of CTAs: cta_group::2 ---------------------------------------------
// Pair tiles of 256 x 256 NW: NW tcgen05 M256 N256 MMAs per K step.  NW = 1
// keeps two 256-column accumulator sets (consecutive tiles, or the two K
// halves of the split forms); NW = 2 fills TMEM with one tile's 512 columns
// and takes in a quarter fewer operand bytes per flop.
template <int NW>
struct PairCfg {
  static constexpr int kStages = NW == 1 ? 6 : 4;
  static constexpr int kABytes = BM * BK * 2;          // this CTA's 128 rows of A: 16 KB
  static constexpr int kBBox = (BN / 2) * BK * 2;      // this CTA's 128 B rows of one N256 MMA: 16 KB
  static constexpr int kBBytes = NW * kBBox;
  static constexpr int kStageBytes = kABytes + kBBytes;
  static constexpr int kTileN = NW * BN;
  static constexpr int kSmemBytes = kStages * kStageBytes + kEpiBytes + 1024 + 256;
};
constexpr int kPairSmemBytes = PairCfg<1>::kSmemBytes;
static_assert(PairCfg<2>::kSmemBytes == kPairSmemBytes, "both pair widths use the same shared memory");
static_assert(kPairSmemBytes <= 232448, "more shared memory than a CTA may have");
// kind::f16, FP32 accumulator, BF16 A and B, both K-major, N = 256, M = 256.
constexpr uint32_t kIdescPair = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                ((uint32_t)((2 * BM) >> 4) << 24);

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release;\n barrier.cluster.wait.acquire;" ::: "memory");
}
// Address of this CTA's shared variable `p` in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_rank(const void *p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// Tile into this CTA's shared memory; the bytes are counted on the mbarrier
// at cluster address `bar` (here: the even CTA's).
__device__ __forceinline__ void tma_load_3d_pair(void *dst, const CUtensorMap *tm, uint32_t bar, int c0, int c1,
                                                 int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cta.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
      " [%0], [%1, {%3, %4, %5}], [%2];"
      ::"r"(smem_u32(dst)), "l"(tm), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
__device__ __forceinline__ void umma_bf16_pair(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(kIdescPair), "r"(accumulate)
      : "memory");
}
// Arrive, once the MMAs issued so far complete, on the mbarrier at the
// offset of `bar` in both CTAs of the pair.
__device__ __forceinline__ void umma_commit_pair_both(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"((uint16_t)3)
      : "memory");
}
__device__ __forceinline__ void umma_commit_pair_local(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// One warp of each CTA of the pair takes part (same columns in both).
__device__ __forceinline__ void tmem_alloc_pair(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Work units of the pair kernel.  Units below `nwhole` are whole tiles; the
// tiles after them (the last, partial wave) are cut along K into `pieces`
// consecutive K-block ranges, one unit each, so that the last wave keeps
// more SMs busy.  Unit u >= nwhole: tile nwhole + (u - nwhole) / pieces, piece
// (u - nwhole) % pieces, K blocks [piece kblocks / pieces, (piece + 1) kblocks / pieces).
struct Unit {
  int t, kb0, nk, slot, piece;                         // slot, piece = -1 for a whole tile
};
__device__ __forceinline__ Unit unit_of(int u, int nwhole, int pieces, int kblocks) {
  Unit w;
  if (u < nwhole) {
    w.t = u;
    w.kb0 = 0;
    w.nk = kblocks;
    w.slot = w.piece = -1;
  } else {
    const int v = u - nwhole;
    w.slot = v / pieces;
    w.piece = v % pieces;
    w.t = nwhole + w.slot;
    w.kb0 = w.piece * kblocks / pieces;
    w.nk = (w.piece + 1) * kblocks / pieces - w.kb0;
  }
  return w;
}

// Product p and K block kb0 + kr of stage j of a unit.  `phased` units run
// in two phases -- the first K half of every product, then the second halves
// -- so that the split forms keep two half sums with one accumulator set.
__device__ __forceinline__ void stage_pk(int j, const Unit &w, int nprod, bool phased, int &p, int &kr) {
  if (!phased) {
    p = j / w.nk;
    kr = j % w.nk;
    return;
  }
  const int h = w.nk / 2, first = nprod * h;
  if (j < first) {
    p = j / h;
    kr = j % h;
  } else {
    const int jj = j - first, h2 = w.nk - h;
    p = jj / h2;
    kr = h + jj % h2;
  }
}
// Launched as clusters of two CTAs; `tm` and `ntiles` count 256 x 256 tiles.
// Pieces of a split tile write FP32 partial tiles to `part` ([slot][piece]
// [8 warps][64][32 lanes] float4: a warp's 32 rows x 256 columns with the
// lanes interleaved, so that every warp access is 512 contiguous bytes); each
// epilogue warp then counts its rows in `cnt` (zeroed before the launch), and
// the warp that arrives last adds the partials in piece order and writes C,
// so the result does not depend on which piece finishes first.  No CTA waits
// for another.
template <int NW>
__global__ void __launch_bounds__(kMmThreads, 1)
    mm_tc_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const __grid_constant__ CUtensorMap tmC, float *__restrict__ C, int64_t M, int64_t N,
                      int64_t ldc, int kblocks, Products prods, TileMap tm, int ntiles, int split_acc, int tma_c,
                      int nwhole, int pieces, float *__restrict__ part, int *__restrict__ cnt,
                      float *__restrict__ halfws) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                          ~uintptr_t(1023));
  using P = PairCfg<NW>;
  unsigned char *sA = smem;
  unsigned char *sB = smem + P::kStages * P::kABytes;
  unsigned char *sEpi = smem + P::kStages * P::kStageBytes;
  uint64_t *full = reinterpret_cast<uint64_t *>(sEpi + kEpiBytes);
  uint64_t *empty = full + P::kStages;
  uint64_t *tfull = empty + P::kStages;
  uint64_t *tempty = tfull + 2;
  uint64_t *mdone = tempty + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mdone + 1);
  volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t crank = cluster_rank();
  const bool leader = crank == 0;
  const int cid = blockIdx.x / 2, ncl = gridDim.x / 2;
  if (threadIdx.x == 0) {
    for (int s = 0; s < P::kStages; ++s) {
      mbar_init(&full[s], 1);                          // even CTA: its producer + both CTAs' bytes
      mbar_init(&empty[s], 1);                         // the even CTA's MMA commit
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 8);                        // even CTA: 4 epilogue warps x 2 CTAs
    }
    mbar_init(mdone, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc_pair(tmem_slot, kTmemCols);
  tc_fence_before();
  cluster_sync();                                      // both CTAs' barriers exist before any remote use
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const bool halves = NW == 1 && split_acc;            // the split forms' two K-half accumulators
  const int nsets = (NW == 1 && !split_acc) ? 2 : 1;
  const int nunits = nwhole + (ntiles - nwhole) * pieces;

  if (warp == 0) {
    if (lane == 0) {                                   // ---- TMA producer (both CTAs)
      int it = 0, issued = 0;
      bool ok = true;
      for (int u = cid; u < nunits && ok; u += ncl) {
        const Unit w = unit_of(u, nwhole, pieces, kblocks);
        int mp, nt;
        tile_coords(w.t, tm, mp, nt);
        // B rows of MMA h: nt * 256 NW + 256 h + (this CTA's half of 256)
        const int arow = mp * 2 * BM + (int)crank * BM, brow = nt * P::kTileN + (int)crank * (BN / 2);
        const int stages = w.nk * prods.n;
        const bool phased = NW == 2 && split_acc && w.nk / 2 > 0;
        for (int j = 0; j < stages; ++j, ++it) {
          const int s = it % P::kStages;
          const uint32_t ph = (it / P::kStages) & 1;
          if (!mbar_wait(&empty[s], ph ^ 1, abort)) { ok = false; break; }
          int p, kr;
          stage_pk(j, w, prods.n, phased, p, kr);
          const int kb = w.kb0 + kr;
          if (leader) mbar_expect_tx(&full[s], 2 * P::kStageBytes);
          const uint32_t fb = map_rank(&full[s], 0);
          tma_load_3d_pair(sA + s * P::kABytes, &tmA, fb, kb * BK, arow, prods.pa[p]);
#pragma unroll
          for (int h = 0; h < NW; ++h)
            tma_load_3d_pair(sB + s * P::kBBytes + h * P::kBBox, &tmB, fb, kb * BK, brow + h * BN, prods.pb[p]);
          issued = it + 1;
        }
      }
      // Before leaving: every issued stage consumed (its MMAs, which read this
      // CTA's shared memory, are done) -- bounded.
      const long long t0 = clock64();
      for (int i = std::max(0, issued - P::kStages); i < issued; ++i)
        while (!mbar_try_wait(&empty[i % P::kStages], (i / P::kStages) & 1) && clock64() - t0 < kWaitBudget) {
        }
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {                         // ---- MMA issuer (even CTA only)
      int it = 0, li = 0;
      bool ok = true, issued_any = false;
      for (int u = cid; u < nunits && ok; u += ncl) {
        const Unit w = unit_of(u, nwhole, pieces, kblocks);
        const int half = w.nk / 2, stages = w.nk * prods.n;
        const bool phased = NW == 2 && split_acc && half > 0;
        int j = 0;
        for (int phz = 0; phz < (phased ? 2 : 1) && ok; ++phz, ++li) {   // one accumulation per phase
          const int si = li % nsets;
          const uint32_t use = (uint32_t)(li / nsets);
          if (!mbar_wait(&tempty[si], (use & 1) ^ 1, abort)) { ok = false; break; }   // both epilogues drained it
          tc_fence_after();
          const int jbeg = j, jend = (phased && phz == 0) ? prods.n * half : stages;
          for (; j < jend; ++j, ++it) {
            const int s = it % P::kStages;
            const uint32_t ph = (it / P::kStages) & 1;
            if (!mbar_wait(&full[s], ph, abort)) { ok = false; break; }
            tc_fence_after();
            int p, kr;                                   // K block kb0 + kr of product p
            stage_pk(j, w, prods.n, phased, p, kr);
            int acc;
            bool first;
            if (halves) {                                // the unit's K range in two halves, one per accumulator
              acc = (half > 0 && kr >= half) ? 1 : 0;
              first = p == 0 && kr == (acc ? half : 0);
            } else {
              acc = si;
              first = j == jbeg;
            }
            const uint32_t d = tmem + (uint32_t)(acc * BN);      // NW = 2: acc = 0, MMA h writes columns 256 h ..
            const uint32_t a0 = smem_u32(sA + s * P::kABytes), b0 = smem_u32(sB + s * P::kBBytes);
#pragma unroll
            for (int k = 0; k < BK / UK; ++k)
#pragma unroll
              for (int h = 0; h < NW; ++h)
                umma_bf16_pair(d + (uint32_t)(h * BN), sdesc(a0 + k * UK * 2), sdesc(b0 + h * P::kBBox + k * UK * 2),
                               (first && k == 0) ? 0u : 1u);
            umma_commit_pair_both(&empty[s]);            // both CTAs' stage s reusable after these MMAs
            issued_any = true;
          }
          if (ok) umma_commit_pair_both(&tfull[si]);     // accumulators complete in both CTAs
        }
      }
      if (issued_any) {                                // every MMA finished before TMEM is freed (bounded)
        umma_commit_pair_local(mdone);
        const long long t0 = clock64();
        while (!mbar_try_wait(mdone, 0) && clock64() - t0 < kWaitBudget) {
        }
      }
    }
  } else {                                             // ---- epilogue, warps 2..5 (both CTAs)
    const int q = warp & 3;                            // TMEM lanes 32 q .. 32 q + 31
    const bool vec = ((ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(C) & 15) == 0);
    const int64_t prow_off = int64_t(crank) * BM + q * 32 + lane;   // this thread's row of a 256-row tile
    constexpr int kChunks = P::kTileN / 32;            // 32-column steps of a row
    const int64_t pstride = int64_t(2 * BM) * P::kTileN / 4;   // one partial tile, in float4
    const int64_t pwarp = (int64_t(crank) * 4 + q) * (32 * P::kTileN / 4) + lane;   // this lane's first float4
    EpiStage es{sEpi + q * 2 * kEpiBufBytes, 0};
    float4 *hrow = halfws ? reinterpret_cast<float4 *>(halfws) + int64_t(cid) * pstride + pwarp : nullptr;
    int li = 0;
    bool stop = false;
    for (int u = cid; u < nunits && !stop; u += ncl) {
      const Unit w = unit_of(u, nwhole, pieces, kblocks);
      const bool two = halves && w.nk / 2 > 0;
      const bool phased = NW == 2 && split_acc && w.nk / 2 > 0;
      int mp, nt;
      tile_coords(w.t, tm, mp, nt);
      const int64_t row = int64_t(mp) * 2 * BM + prow_off;
      const int64_t n0 = int64_t(nt) * P::kTileN;
      float4 *prow = w.piece >= 0
                         ? reinterpret_cast<float4 *>(part) + (int64_t(w.slot) * pieces + w.piece) * pstride + pwarp
                         : nullptr;
      for (int phz = 0; phz < (phased ? 2 : 1); ++phz, ++li) {
        const int si = li % nsets;
        const uint32_t use = (uint32_t)(li / nsets);
        if (!mbar_wait(&tfull[si], use & 1, abort)) { stop = true; break; }
        tc_fence_after();
        const bool keep = phased && phz == 0;           // the first K half: kept for the second phase
        const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(nsets == 2 ? si * BN : 0);
#pragma unroll 1
        for (int c = 0; c < kChunks; ++c) {
          uint32_t r[32];
          tmem_ld32(base + (uint32_t)(c * 32), r);
          if (keep) {                                    // this lane's own slots: read back by it alone
#pragma unroll
            for (int j = 0; j < 8; ++j)
              __stcg(hrow + (c * 8 + j) * 32,
                   make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]), __uint_as_float(r[4 * j + 2]),
                               __uint_as_float(r[4 * j + 3])));
            continue;
          }
          if (phased) {                                  // first half + second half, as the two accumulators add
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const float4 v = __ldcg(hrow + (c * 8 + j) * 32);
              r[4 * j] = __float_as_uint(__fadd_rn(v.x, __uint_as_float(r[4 * j])));
              r[4 * j + 1] = __float_as_uint(__fadd_rn(v.y, __uint_as_float(r[4 * j + 1])));
              r[4 * j + 2] = __float_as_uint(__fadd_rn(v.z, __uint_as_float(r[4 * j + 2])));
              r[4 * j + 3] = __float_as_uint(__fadd_rn(v.w, __uint_as_float(r[4 * j + 3])));
            }
          } else if (two) {
            uint32_t r1[32];
            tmem_ld32(base + (uint32_t)(BN + c * 32), r1);
#pragma unroll
            for (int j = 0; j < 32; ++j)
              r[j] = __float_as_uint(__fadd_rn(__uint_as_float(r[j]), __uint_as_float(r1[j])));
          }
          if (prow) {                                    // a piece: the partial tile, kept in L2
#pragma unroll
            for (int j = 0; j < 8; ++j)
              __stcg(prow + (c * 8 + j) * 32,
                     make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                 __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3])));
          } else if (tma_c) {
            epi_store_box(es, &tmC, (int)(n0 + c * 32), (int)(row - lane), row - lane < M && n0 + c * 32 < N, lane, r);
          } else {
            store_row32(C, row, n0 + c * 32, M, N, ldc, vec, r);
          }
        }
        tc_fence_before();                               // TMEM reads done before the set is reused
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(map_rank(&tempty[si], 0));
      }
      if (stop) break;
      if (prow) {                                      // the last piece to arrive writes C
        __threadfence();
        __syncwarp();
        int seen = 0;
        if (lane == 0) seen = atomicAdd(&cnt[w.slot * 8 + (int)crank * 4 + q], 1);
        seen = __shfl_sync(0xffffffffu, seen, 0);
        if (seen == pieces - 1) {
          __threadfence();
          const float4 *p0 = reinterpret_cast<const float4 *>(part) + int64_t(w.slot) * pieces * pstride + pwarp;
#pragma unroll 1
          for (int c = 0; c < kChunks; c += 2) {       // 64 columns: 16 loads in flight per piece
            float4 a[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) a[j] = __ldcg(p0 + (c * 8 + j) * 32);
#pragma unroll 1
            for (int pc = 1; pc < pieces; ++pc) {
              float4 b[16];
#pragma unroll
              for (int j = 0; j < 16; ++j) b[j] = __ldcg(p0 + pc * pstride + (c * 8 + j) * 32);
#pragma unroll
              for (int j = 0; j < 16; ++j)
                a[j] = make_float4(__fadd_rn(a[j].x, b[j].x), __fadd_rn(a[j].y, b[j].y), __fadd_rn(a[j].z, b[j].z),
                                   __fadd_rn(a[j].w, b[j].w));
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              uint32_t r[32];
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                r[4 * j] = __float_as_uint(a[8 * h + j].x);
                r[4 * j + 1] = __float_as_uint(a[8 * h + j].y);
                r[4 * j + 2] = __float_as_uint(a[8 * h + j].z);
                r[4 * j + 3] = __float_as_uint(a[8 * h + j].w);
              }
              const int64_t col = n0 + (c + h) * 32;
              if (tma_c)
                epi_store_box(es, &tmC, (int)col, (int)(row - lane), row - lane < M && col < N, lane, r);
              else
                store_row32(C, row, col, M, N, ldc, vec, r);
            }
          }
        }
      }
    }
    epi_drain(lane);
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();                                      // both CTAs done with TMEM and each other's barriers
  if (warp == 1) tmem_dealloc_pair(tmem, kTmemCols);
  cluster_sync();                                      // neither CTA of the pair leaves first
}

// ---- split pass: FP32 source (any 2-D strides) -> P BF16 planes, zero padded
// Output plane p is R x Cc row-major (padded to Rp x Cp); element (r, c) of
// the logical source is src[off + r * sr + c * sc].  Planes: p = 0 holds
// bf16(x), p = 1 bf16(x - x0), p = 2 bf16(x - x0 - x1) (FP32 differences).
// Three kernels, by the source's layout: columns contiguous (no transposition,
// 8 elements per thread, 16-byte loads and stores), rows contiguous (64 x 64
// tiles transposed through shared memory), and any other strides.
constexpr int kTT = 64;

// The planes of 8 consecutive values, 8 BF16 (16 bytes) per plane.
__device__ __forceinline__ void split8(const float (&x)[8], uint4 (&o)[3]) {
  uint32_t w[3][4];
#pragma unroll
  for (int k = 0; k < 8; k += 2) {
    __nv_bfloat16 h[3][2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const __nv_bfloat16 a0 = __float2bfloat16_rn(x[k + e]);
      const float r1 = __fsub_rn(x[k + e], __bfloat162float(a0));
      const __nv_bfloat16 a1 = __float2bfloat16_rn(r1);
      const float r2 = __fsub_rn(r1, __bfloat162float(a1));
      h[0][e] = a0;
      h[1][e] = a1;
      h[2][e] = __float2bfloat16_rn(r2);
    }
#pragma unroll
    for (int p = 0; p < 3; ++p)
      w[p][k / 2] = (uint32_t)__bfloat16_as_ushort(h[p][0]) | ((uint32_t)__bfloat16_as_ushort(h[p][1]) << 16);
  }
#pragma unroll
  for (int p = 0; p < 3; ++p) o[p] = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
}

// sc == 1 and 16-byte aligned rows: a thread takes 8 columns of one row, two
// such chunks per step (both loaded before either is split).
__device__ __forceinline__ void load8(const float *__restrict__ src, int64_t off, int64_t sr, int64_t R,
                                      int64_t Cc, int64_t r, int64_t c, float (&x)[8]) {
  if (r < R && c + 8 <= Cc) {
    const float4 *q = reinterpret_cast<const float4 *>(src + off + r * sr + c);
    const float4 a = __ldcs(q), b = __ldcs(q + 1);
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (r < R && c + j < Cc) ? src[off + r * sr + c + j] : 0.f;
  }
}
// The planes of x into rows r of each plane, columns c .. c + 7.
__device__ __forceinline__ void store8(__nv_bfloat16 *__restrict__ dst, int64_t Rp, int64_t Cp, int planes,
                                       int64_t r, int64_t c, const float (&x)[8]) {
  uint4 o[3];
  split8(x, o);
#pragma unroll
  for (int p = 0; p < 3; ++p)
    if (p < planes) *reinterpret_cast<uint4 *>(dst + (int64_t(p) * Rp + r) * Cp + c) = o[p];
}
// Block 0 of each split kernel also zeroes `clear[0, nclear)` (the matmul's
// piece counters), which saves a launch.
__device__ __forceinline__ void clear_words(int *clear, int nclear) {
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < nclear; i += blockDim.x) clear[i] = 0;
}
__global__ void __launch_bounds__(256) split_rows_kernel(const float *__restrict__ src, int64_t off, int64_t sr,
                                                         int64_t R, int64_t Cc, int64_t Rp, int64_t Cp, int planes,
                                                         __nv_bfloat16 *__restrict__ dst, int *clear, int nclear) {
  clear_words(clear, nclear);
  const int64_t per_row = Cp / 8, total = Rp * per_row;
  const int64_t stride = int64_t(gridDim.x) * 256;
  for (int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x; i < total; i += 2 * stride) {
    const int64_t i2 = i + stride;
    const int64_t r = i / per_row, c = (i - r * per_row) * 8;
    const int64_t r2 = i2 / per_row, c2 = (i2 - r2 * per_row) * 8;
    float x[8], y[8];
    load8(src, off, sr, R, Cc, r, c, x);
    if (i2 < total) load8(src, off, sr, R, Cc, r2, c2, y);
    store8(dst, Rp, Cp, planes, r, c, x);
    if (i2 < total) store8(dst, Rp, Cp, planes, r2, c2, y);
  }
}

// sr == 1 (rows contiguous: the source is the transpose of the planes'
// layout), 16-byte aligned columns: 64 x 64 tiles through shared memory,
// read as float4 along r, written as 8 BF16 along c.  Persistent: a CTA walks
// tiles blockIdx.x, blockIdx.x + gridDim.x, ..., and the loads of its next
// tile are in flight while the current one is split and stored.
__device__ __forceinline__ void split_cols_load(const float *__restrict__ src, int64_t off, int64_t sc, int64_t R,
                                                int64_t Cc, int64_t r0, int64_t c0, int tid, float4 (&v)[4]) {
#pragma unroll
  for (int i = 0; i < kTT * kTT / 4 / 256; ++i) {
    const int f = i * 256 + tid;
    const int lc = f / (kTT / 4), lr = (f % (kTT / 4)) * 4;
    const int64_t r = r0 + lr, c = c0 + lc;
    if (c < Cc && r + 4 <= R) {
      v[i] = __ldcs(reinterpret_cast<const float4 *>(src + off + r + c * sc));
    } else {
      float e[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) e[j] = (c < Cc && r + j < R) ? src[off + r + j + c * sc] : 0.f;
      v[i] = make_float4(e[0], e[1], e[2], e[3]);
    }
  }
}
__global__ void __launch_bounds__(256, 6) split_cols_kernel(const float *__restrict__ src, int64_t off, int64_t sc,
                                                         int64_t R, int64_t Cc, int64_t Rp, int64_t Cp, int planes,
                                                         __nv_bfloat16 *__restrict__ dst, int *clear, int nclear) {
  clear_words(clear, nclear);
  __shared__ float tile[kTT][kTT + 1];                 // [c][r]
  const int tid = threadIdx.x;
  const int64_t tiles_c = Cp / kTT, ntiles = (Rp / kTT) * tiles_c;
  int64_t t = blockIdx.x;
  float4 v[4];
  if (t < ntiles) split_cols_load(src, off, sc, R, Cc, (t / tiles_c) * kTT, (t % tiles_c) * kTT, tid, v);
  for (; t < ntiles; t += gridDim.x) {
    const int64_t r0 = (t / tiles_c) * kTT, c0 = (t % tiles_c) * kTT;
    __syncthreads();                                   // the previous tile's shared reads are done
#pragma unroll
    for (int i = 0; i < kTT * kTT / 4 / 256; ++i) {
      const int f = i * 256 + tid;
      const int lc = f / (kTT / 4), lr = (f % (kTT / 4)) * 4;
      tile[lc][lr] = v[i].x;
      tile[lc][lr + 1] = v[i].y;
      tile[lc][lr + 2] = v[i].z;
      tile[lc][lr + 3] = v[i].w;
    }
    __syncthreads();
    const int64_t tn = t + gridDim.x;
    if (tn < ntiles) split_cols_load(src, off, sc, R, Cc, (tn / tiles_c) * kTT, (tn % tiles_c) * kTT, tid, v);
#pragma unroll
    for (int i = 0; i < kTT * kTT / 8 / 256; ++i) {
      const int e = i * 256 + tid;
      const int lr = e / (kTT / 8), lc = (e % (kTT / 8)) * 8;
      float x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = tile[lc + j][lr];
      store8(dst, Rp, Cp, planes, r0 + lr, c0 + lc, x);
    }
  }
}

// Any strides: 64 x 64 tiles, element loads in the direction of the smaller
// stride.
__global__ void __launch_bounds__(256) split_planes_kernel(const float *__restrict__ src, int64_t off, int64_t sr,
                                                           int64_t sc, int64_t R, int64_t Cc, int64_t Rp,
                                                           int64_t Cp, int planes,
                                                           __nv_bfloat16 *__restrict__ dst, int *clear, int nclear) {
  clear_words(clear, nclear);
  __shared__ float tile[kTT][kTT + 1];
  const int tid = threadIdx.x;
  const int64_t tiles_c = Cp / kTT;
  const int64_t r0 = (int64_t(blockIdx.x) / tiles_c) * kTT, c0 = (int64_t(blockIdx.x) % tiles_c) * kTT;
  const bool rows_contig = (sr == 1 && sc != 1);        // read along r for coalescing
#pragma unroll 4
  for (int i = 0; i < kTT * kTT / 256; ++i) {
    const int e = i * 256 + tid;
    const int lr = rows_contig ? (e % kTT) : (e / kTT);
    const int lc = rows_contig ? (e / kTT) : (e % kTT);
    const int64_t r = r0 + lr, c = c0 + lc;
    tile[lr][lc] = (r < R && c < Cc) ? src[off + r * sr + c * sc] : 0.f;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kTT * kTT / 8 / 256; ++i) {
    const int e = i * 256 + tid;
    const int lr = e / (kTT / 8), lc = (e % (kTT / 8)) * 8;
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = tile[lr][lc + j];
    store8(dst, Rp, Cp, planes, r0 + lr, c0 + lc, x);
  }
}

// Planes of one operand; Rp and Cp are multiples of 64.
int32_t launch_split(const float *src, int64_t off, int64_t sr, int64_t sc, int64_t R, int64_t Cc, int64_t Rp,
                     int64_t Cp, int planes, __nv_bfloat16 *dst, cudaStream_t s, int nsm, int *clear = nullptr,
                     int nclear = 0) {
  const bool base16 = ((reinterpret_cast<uintptr_t>(src + off)) & 15) == 0;
  const int64_t tiles = (Rp / kTT) * (Cp / kTT);
  if (sc == 1 && base16 && (sr & 3) == 0) {
    const int64_t blocks = std::min<int64_t>((Rp * (Cp / 8) + 255) / 256, int64_t(nsm) * 64);
    split_rows_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(src, off, sr, R, Cc, Rp, Cp, planes,
                                                                            dst, clear, nclear);
  } else {
    if (tiles >= (int64_t(1) << 31)) return DESC_ERR_UNSUPPORTED;
    if (sr == 1 && base16 && (sc & 3) == 0)
      split_cols_kernel<<<(unsigned)std::min<int64_t>(tiles, int64_t(nsm) * 6), 256, 0, s>>>(   // 6 resident per SM
          src, off, sc, R, Cc, Rp, Cp, planes, dst, clear, nclear);
    else
      split_planes_kernel<<<(unsigned)tiles, 256, 0, s>>>(src, off, sr, sc, R, Cc, Rp, Cp, planes, dst, clear,
                                                          nclear);
  }
  DESC_CUDA_TRY(cudaGetLastError());
  return DESC_OK;
}

// ---- tensor maps -----------------------------------------------------------
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

// [planes][rows][cols] BF16, box = box_rows x 64 columns x 1 plane.
bool make_map(CUtensorMap *m, const void *base, int64_t planes, int64_t rows, int64_t cols, int box_rows) {
  EncodeTiled enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)(cols * 2), (cuuint64_t)(rows * cols * 2)};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C (M x N FP32, rows ldc apart) for the epilogue's TMA stores: 32 x 32
// boxes, 128-byte swizzle.  false where TMA cannot address C (base not 16-byte
// aligned, row pitch not a multiple of 16 bytes, extents of 2^31 or more);
// the epilogue then stores from registers.
bool make_map_c(CUtensorMap *m, float *C, int64_t M, int64_t N, int64_t ldc) {
  EncodeTiled enc = encoder();
  if (!enc || (reinterpret_cast<uintptr_t>(C) & 15) != 0 || (ldc & 3) != 0 || M >= (int64_t(1) << 31) ||
      N >= (int64_t(1) << 31))
    return false;
  cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)M};
  cuuint64_t strides[1] = {(cuuint64_t)(ldc * 4)};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, C, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// Schedule candidates (candidates.h): 0 pairs (where the tile rows pair up),
// wide groups; 1 single CTAs, wide groups; 2 pairs, narrow groups; 3 single,
// narrow; 4 / 5 pairs with 256 x 512 tiles, wide / narrow groups.
constexpr int kMmCandCount = kNumMmCands;
static_assert(kMmCands[0].group_rows == kGroupM, "the default candidate uses the wide groups");

int mm_candidates() { return kMmCandCount; }
void mm_candidate(int cand, int *pairs, int *group_rows, int *width) {
  const MmCand &c = kMmCands[(cand >= 0 && cand < kMmCandCount) ? cand : 0];
  *pairs = c.pairs;
  *group_rows = c.group_rows;
  if (width) *width = c.width;
}

int32_t mm_status_take() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_mm_status, sizeof(int)) != cudaSuccess) return DESC_ERR_CUDA;
  if (v != 0 && cudaMemcpyToSymbol(g_mm_status, &z, sizeof(int)) != cudaSuccess) return DESC_ERR_CUDA;
  return v;
}

namespace {

// One product: odd 128-row tile counts from this one up are padded to pair
// up (measured on GB300, N = K = 4096: 3 to 7 tile rows ran 1-6 % slower
// padded, 15 rows 2-7 % faster, M = 8064 at 8192^2 14 % faster; the split
// forms ran faster padded at every count, M = 8064 by 22 %).
constexpr int kMinPadRowsBF16 = 9;
constexpr int kMaxPieces = 4;         // K pieces per tile of the last wave
// Stages (K blocks of 64 x products) per piece, at least: a piece costs a
// partial-tile round trip through L2 and the final sum, which pays off only
// when it saves more MMA time than that (measured on GB300: BF16 products
// lost with 12 stages per piece and gained with 32).
constexpr int kMinPieceStages = 24;
constexpr size_t kPartTileBytes = size_t(2 * BM) * PairCfg<2>::kTileN * 4;   // the wider pair tile

struct MmDevice {
  int32_t status = DESC_ERR_CUDA;
  int nsm = 0, max_pairs = 0;
};

// Kernel attributes, SM count and the number of CTA pairs resident at once
// (an SM without a partner in its GPC stays idle), once per device (kernel
// attributes belong to the device that is current when they are set).
constexpr int kMaxDevices = 64;
const MmDevice &mm_device() {
  static MmDevice per_dev[kMaxDevices];
  static std::once_flag once[kMaxDevices];
  static const MmDevice none;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return none;
  MmDevice &d = per_dev[dev];
  std::call_once(once[dev], [&d, dev] {
    if (cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(mm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess ||
        cudaFuncSetAttribute(mm_tc_pair_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPairSmemBytes) !=
            cudaSuccess ||
        cudaFuncSetAttribute(mm_tc_pair_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPairSmemBytes) !=
            cudaSuccess)
      return;
    cudaLaunchConfig_t q{};
    cudaLaunchAttribute qa[1];
    qa[0].id = cudaLaunchAttributeClusterDimension;
    qa[0].val.clusterDim.x = 2;
    qa[0].val.clusterDim.y = 1;
    qa[0].val.clusterDim.z = 1;
    q.gridDim = dim3(2 * (unsigned)std::max(d.nsm / 2, 1));
    q.blockDim = dim3(kMmThreads);
    q.dynamicSmemBytes = kPairSmemBytes;
    q.attrs = qa;
    q.numAttrs = 1;
    int wide_pairs = 0;
    if (cudaOccupancyMaxActiveClusters(&d.max_pairs, mm_tc_pair_kernel<1>, &q) != cudaSuccess ||
        cudaOccupancyMaxActiveClusters(&wide_pairs, mm_tc_pair_kernel<2>, &q) != cudaSuccess)
      return;
    d.max_pairs = std::min(d.max_pairs, wide_pairs);
    d.status = DESC_OK;
  });
  return d;
}

// How the pair kernel cuts the last wave: tiles [0, *full) whole, the rest
// in *pieces K ranges.  ntiles counts 256 x 256 tiles.
void pair_units(int64_t ntiles, int kblocks, int nprod, int max_pairs, int64_t *full, int *pieces) {
  *full = ntiles;
  *pieces = 1;
  if (max_pairs < 1) return;
  const int64_t tail = ntiles % max_pairs;
  if (tail == 0) return;
  const int pc =
      (int)std::min<int64_t>({kMaxPieces, max_pairs / tail, int64_t(kblocks) * nprod / kMinPieceStages});
  if (pc < 2) return;
  *full = ntiles - tail;
  *pieces = pc;
}

// Room for the split forms' first K halves of 512-wide tiles (one tile per
// resident pair), then the partial tiles and counters of the pieces (at most
// one partial tile per resident pair).
size_t half_bytes(int planes) {
  const int mp = mm_device().max_pairs;
  return planes > 1 && mp > 0 ? align256(size_t(mp) * kPartTileBytes) : 0;
}
size_t part_bytes(int64_t M, int64_t N, int planes) {
  const int64_t Mp = round_up(M, 2 * BM), Np = round_up(N, BN);   // tile rows padded to pair up
  const int mp = mm_device().max_pairs;
  const int64_t ntiles = (Mp / (2 * BM)) * (Np / BN);
  const int64_t slots = std::min<int64_t>(mp, ntiles * kMaxPieces);
  return half_bytes(planes) +
         (slots > 0 ? align256(size_t(slots) * kPartTileBytes) + align256(size_t(mp) * 8 * sizeof(int)) : 0);
}

}  // namespace

// Planes needed by a precision: 1 (BF16), 2 (2-term split), 3 (3-term split),
// then the pieces' partial tiles.
int mm_max_pairs() {
  const MmDevice &d = mm_device();
  return d.status == DESC_OK ? d.max_pairs : 0;
}

int32_t mm_plan(int64_t M, int64_t N, int64_t K, int nprod, int cand, int max_pairs, MmPlan *pl) {
  if (!pl || M <= 0 || N <= 0 || K <= 0 || nprod < 1 || cand >= kMmCandCount) return DESC_ERR_INVALID_ARG;
  const int64_t Mp1 = round_up(M, BM), Mp2 = round_up(M, 2 * BM), Np = round_up(N, BN), Kp = round_up(K, BK);
  if (Mp2 / BM > 65535 || Np / BN > (int64_t(1) << 30) || Kp > (int64_t(1) << 30)) return DESC_ERR_UNSUPPORTED;
  // Untuned: 256 x 512 pair tiles where they fill at least half of the
  // resident pairs for one product, a quarter for the split forms (measured on
  // GB300: SPLIT3 8192^3 4.32 -> 3.63 ms, 4096^3 0.615 -> 0.542 ms, 640 x 4096^2
  // 198 -> 162 us with 24 wide tiles; BF16 8192^3 756 -> 728 us, but at 2048^3,
  // 32 wide tiles, BF16 42 -> 50 us, and SPLIT3 111 -> 113 us), else 256 x 256.
  if (cand < 0) {
    const int64_t wide_tiles = (Mp2 / (2 * BM)) * ((Np + 2 * BN - 1) / (2 * BN));
    cand = (nprod > 1 ? 4 * wide_tiles : 2 * wide_tiles) >= max_pairs ? 4 : 0;
  }
  int want_pairs = 1, group_rows = kGroupM, width = 1;
  mm_candidate(cand, &want_pairs, &group_rows, &width);
  // CTA pairs over 256 x 256 (or 256 x 512) tiles (cta_group::2), else single
  // CTAs over 128 x 256 tiles.  An odd count of 128-row tiles is padded with
  // one zero tile row (the split pass writes zeros there, the epilogue stores
  // no row past M) where the pairs' leaner operand stream pays for the extra row.
  const bool pad = want_pairs && max_pairs >= 1 && (Mp1 / BM) % 2 == 1 && (nprod > 1 || Mp1 / BM >= kMinPadRowsBF16);
  const int64_t Mp = pad ? Mp2 : Mp1;
  const bool pairs = want_pairs && (Mp / BM) % 2 == 0 && max_pairs >= 1;
  if (!pairs) width = 1;
  pl->cand = cand;
  pl->pairs = pairs ? 1 : 0;
  pl->width = width;
  pl->padded = pad ? 1 : 0;
  pl->group_rows = group_rows;
  pl->Mp = Mp;
  pl->tiles_m = pairs ? Mp / (2 * BM) : Mp / BM;
  pl->tiles_n = (Np + BN * width - 1) / (BN * width);
  pl->tiles = pl->tiles_m * pl->tiles_n;
  if (pl->tiles >= (int64_t(1) << 31)) return DESC_ERR_UNSUPPORTED;
  pl->whole = pl->tiles;
  pl->pieces = 1;
  if (pairs) {
    pair_units(pl->tiles, (int)(Kp / BK), nprod, max_pairs, &pl->whole, &pl->pieces);
    if (pl->whole + (pl->tiles - pl->whole) * pl->pieces >= (int64_t(1) << 31)) return DESC_ERR_UNSUPPORTED;
  }
  return DESC_OK;
}

// The A planes have room for an even number of 128-row tiles (an odd count
// may be padded with a zero tile row so that the rows pair up).
size_t mm_tc_ws(int64_t M, int64_t N, int64_t K, int planes) {
  const int64_t Mp = round_up(M, 2 * BM), Np = round_up(N, BN), Kp = round_up(K, BK);
  return align256(size_t(planes) * Mp * Kp * 2) + align256(size_t(planes) * Np * Kp * 2) + part_bytes(M, N, planes);
}

int32_t launch_mm_tc(const float *A, int64_t a_off, int64_t a_sr, int64_t a_sc, const float *B, int64_t b_off,
                     int64_t b_sr, int64_t b_sc, float *C, int64_t M, int64_t N, int64_t K, int planes,
                     int nprod, const int *pa, const int *pb, void *ws, size_t ws_bytes, desc_stream_t st) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  const int64_t Mp2 = round_up(M, 2 * BM), Np = round_up(N, BN), Kp = round_up(K, BK);
  if (!ws || ws_bytes < mm_tc_ws(M, N, K, planes)) return DESC_ERR_WORKSPACE;
  if (Mp2 / BM > 65535 || Np / BN > (int64_t(1) << 30) || Kp > (int64_t(1) << 30)) return DESC_ERR_UNSUPPORTED;
  const MmDevice &dv = mm_device();
  if (dv.status != DESC_OK) return dv.status;
  const int nsm = dv.nsm, max_pairs = dv.max_pairs;
  __nv_bfloat16 *pA = static_cast<__nv_bfloat16 *>(ws);
  __nv_bfloat16 *pB = reinterpret_cast<__nv_bfloat16 *>(static_cast<char *>(ws) +
                                                         align256(size_t(planes) * Mp2 * Kp * 2));
  char *pbase = static_cast<char *>(ws) + align256(size_t(planes) * Mp2 * Kp * 2) +
                align256(size_t(planes) * Np * Kp * 2);
  MmPlan pl;
  int32_t r = mm_plan(M, N, K, nprod, schedule_for(DESC_OP_MATMUL, DESC_F32, M, N), max_pairs, &pl);
  if (r != DESC_OK) return r;
  const bool pairs = pl.pairs != 0;
  const int width = pl.width;
  const int64_t Mp = pl.Mp, ntiles = pl.tiles, nwhole = pl.whole;
  const int pieces = pl.pieces;
  TileMap tmap;
  tmap.Mt = (int)pl.tiles_m;
  tmap.Nt = (int)pl.tiles_n;
  tmap.group_m = std::min(tmap.Mt, pairs ? pl.group_rows / 2 : pl.group_rows);
  const int kblocks = (int)(Kp / BK), split = planes > 1 ? 1 : 0;
  float *part = nullptr;
  int *cnt = nullptr;
  int ncnt = 0;
  if (pieces > 1) {
    const int64_t slots = ntiles - nwhole;
    part = reinterpret_cast<float *>(pbase + half_bytes(planes));
    cnt = reinterpret_cast<int *>(pbase + half_bytes(planes) + align256(size_t(slots * pieces) * kPartTileBytes));
    ncnt = (int)(slots * 8);
  }

  // A (M x K) -> planes [P][Mp][Kp];  B (K x N) -> transposed planes [P][Np][Kp];
  // the A pass also zeroes the pieces' counters.
  r = launch_split(A, a_off, a_sr, a_sc, M, K, Mp, Kp, planes, pA, s, nsm, cnt, ncnt);
  if (r != DESC_OK) return r;
  r = launch_split(B, b_off, b_sc, b_sr, N, K, Np, Kp, planes, pB, s, nsm);
  if (r != DESC_OK) return r;
  CUtensorMap tmA, tmB, tmC{};
  if (!make_map(&tmA, pA, planes, Mp, Kp, BM) || !make_map(&tmB, pB, planes, Np, Kp, pairs ? BN / 2 : BN))
    return DESC_ERR_CUDA;
  const int tma_c = make_map_c(&tmC, C, M, N, N) ? 1 : 0;
  Products pr{};
  pr.n = nprod;
  for (int i = 0; i < nprod; ++i) {
    pr.pa[i] = pa[i];
    pr.pb[i] = pb[i];
  }
  if (!pairs) {
    const int grid = (int)std::min<int64_t>(ntiles, std::max(nsm, 1));
    mm_tc_kernel<<<grid, kMmThreads, kSmemBytes, s>>>(tmA, tmB, tmC, C, M, N, N, kblocks, pr, tmap, (int)ntiles, split,
                                                      tma_c);
  } else {
    const int64_t nunits = nwhole + (ntiles - nwhole) * pieces;
    const int npairs = (int)std::min<int64_t>(nunits, max_pairs);
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute la[1];
    la[0].id = cudaLaunchAttributeClusterDimension;
    la[0].val.clusterDim.x = 2;
    la[0].val.clusterDim.y = 1;
    la[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * (unsigned)npairs);
    cfg.blockDim = dim3(kMmThreads);
    cfg.dynamicSmemBytes = kPairSmemBytes;
    cfg.stream = s;
    cfg.attrs = la;
    cfg.numAttrs = 1;
    float *halfws = (width == 2 && split) ? reinterpret_cast<float *>(pbase) : nullptr;
    if (width == 2)
      DESC_CUDA_TRY(cudaLaunchKernelEx(&cfg, mm_tc_pair_kernel<2>, tmA, tmB, tmC, C, M, N, N, kblocks, pr, tmap,
                                       (int)ntiles, split, tma_c, (int)nwhole, pieces, part, cnt, halfws));
    else
      DESC_CUDA_TRY(cudaLaunchKernelEx(&cfg, mm_tc_pair_kernel<1>, tmA, tmB, tmC, C, M, N, N, kblocks, pr, tmap,
                                       (int)ntiles, split, tma_c, (int)nwhole, pieces, part, cnt, halfws));
  }
  DESC_CUDA_TRY(cudaGetLastError());
  return DESC_OK;
}

}  // namespace desc
