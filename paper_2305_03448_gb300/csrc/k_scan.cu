// Inclusive (and exclusive) scans: sums, maxima and minima over contiguous
// runs, per-level segments and CSR segments -- the single-pass look-back scan
// of k_scan_core.cuh -- and the entry points that route the other operators
// and the other schedules to the units that compile them.
#include "k_scan_core.cuh"

namespace desc {

namespace {
constexpr int32_t kOtherValueOps = DESC_PROD | DESC_AND | DESC_OR | DESC_XOR;
}  // namespace

int32_t scan_status_take() {
  // every unit's word is read (and cleared); the first error is reported
  const int32_t w[6] = {take_status_word(), scan_status_take_ops(), scan_status_take_mapped(),
                        scan_status_take_mapped2(), scan_status_take_argmap(), scan_status_take_map()};
  for (int32_t v : w)
    if (v != DESC_OK) return v;
  return DESC_OK;
}

size_t scan_contig_ws(int32_t /*dtype*/, int64_t n) {
  const int64_t ntiles = (n + kWsTile - 1) / kWsTile;
  return align256(sizeof(ScanWs)) + size_t(ntiles) * sizeof(TileState);
}

int scan_candidates() { return kNumScanCands; }

size_t scan_csr_ws(int64_t n) { return scan_contig_ws(DESC_F32, n); }

int32_t launch_scan_contig(int32_t dtype, const void *in, void *out, int64_t n, int64_t period,
                           int32_t flags, void *ws, size_t ws_bytes, desc_stream_t st, int cand) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  ScanArgs a{};
  a.n = n;
  a.period = period;
  a.debug = (flags & DESC_DEBUG_STALL_TILE) ? 1 : 0;
  a.vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
  const bool periodic = period > 0 && period < n;
  const MapArgs none{};
  if (flags & kOtherValueOps) return launch_scan_contig_ops(dtype, in, out, n, period, flags, ws, ws_bytes, st);
  if (dtype == DESC_I32) {
    auto i = static_cast<const int32_t *>(in);
    auto o = static_cast<int32_t *>(out);
    return periodic ? run_scan_basic<int32_t, PERIODIC, false>(i, o, a, ws, ws_bytes, s, cand, flags, none)
                    : run_scan_basic<int32_t, PLAIN, false>(i, o, a, ws, ws_bytes, s, cand, flags, none);
  }
  auto i = static_cast<const float *>(in);
  auto o = static_cast<float *>(out);
  return periodic ? run_scan_basic<float, PERIODIC, false>(i, o, a, ws, ws_bytes, s, cand, flags, none)
                  : run_scan_basic<float, PLAIN, false>(i, o, a, ws, ws_bytes, s, cand, flags, none);
}

int32_t launch_scan_csr(int32_t dtype, const void *in, void *out, int64_t n, const int64_t *offsets,
                        int64_t nseg, void *sums, int32_t flags, void *ws, size_t ws_bytes,
                        desc_stream_t st, int cand) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  const SegCand sc = kSegCands[(cand >= 0 && cand < kNumSegCands) ? cand : 0];
  if (sc.threads > 0 && !(flags & DESC_DEBUG_STALL_TILE) && !(flags & kOtherValueOps))   // a group per segment
    return launch_seg_group(dtype, in, out, offsets, nseg, sums, flags, sc.threads, st);
  if (flags & kOtherValueOps) return launch_scan_csr_ops(dtype, in, out, n, offsets, nseg, sums, flags, ws, ws_bytes, st);
  if (sc.threads == 0) cand = cand >= 0 && cand < kNumScanCands ? cand : 0;   // tiles of 4096 x sub
  ScanArgs a{};
  a.n = n;
  a.offsets = offsets;
  a.nseg = nseg;
  a.sums = sums;
  a.debug = (flags & DESC_DEBUG_STALL_TILE) ? 1 : 0;
  a.vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
  const MapArgs none{};
  if (dtype == DESC_I32)
    return run_scan_basic<int32_t, CSR, false>(static_cast<const int32_t *>(in), static_cast<int32_t *>(out), a,
                                  ws, ws_bytes, s, cand, flags, none);
  return run_scan_basic<float, CSR, false>(static_cast<const float *>(in), static_cast<float *>(out), a, ws,
                              ws_bytes, s, cand, flags, none);
}

}  // namespace desc
