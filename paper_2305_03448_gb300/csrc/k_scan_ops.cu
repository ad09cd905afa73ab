// Scans with the product and the bitwise operators (the look-back scan of
// k_scan_core.cuh over contiguous runs, per-level segments and CSR segments).
#include "k_scan_core.cuh"

namespace desc {

int32_t scan_status_take_ops() { return take_status_word(); }

int32_t launch_scan_contig_ops(int32_t dtype, const void *in, void *out, int64_t n, int64_t period, int32_t flags,
                               void *ws, size_t ws_bytes, desc_stream_t st) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  ScanArgs a{};
  a.n = n;
  a.period = period;
  a.debug = (flags & DESC_DEBUG_STALL_TILE) ? 1 : 0;
  a.vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
  const bool periodic = period > 0 && period < n;
  const MapArgs none{};
  if (dtype == DESC_I32) {
    auto i = static_cast<const int32_t *>(in);
    auto o = static_cast<int32_t *>(out);
    return periodic ? run_scan_ops<int32_t, PERIODIC, false>(i, o, a, ws, ws_bytes, s, flags, none)
                    : run_scan_ops<int32_t, PLAIN, false>(i, o, a, ws, ws_bytes, s, flags, none);
  }
  auto i = static_cast<const float *>(in);
  auto o = static_cast<float *>(out);
  return periodic ? run_scan_ops<float, PERIODIC, false>(i, o, a, ws, ws_bytes, s, flags, none)
                  : run_scan_ops<float, PLAIN, false>(i, o, a, ws, ws_bytes, s, flags, none);
}

int32_t launch_scan_csr_ops(int32_t dtype, const void *in, void *out, int64_t n, const int64_t *offsets,
                            int64_t nseg, void *sums, int32_t flags, void *ws, size_t ws_bytes, desc_stream_t st) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  ScanArgs a{};
  a.n = n;
  a.offsets = offsets;
  a.nseg = nseg;
  a.sums = sums;
  a.debug = (flags & DESC_DEBUG_STALL_TILE) ? 1 : 0;
  a.vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
  const MapArgs none{};
  if (dtype == DESC_I32)
    return run_scan_ops<int32_t, CSR, false>(static_cast<const int32_t *>(in), static_cast<int32_t *>(out), a, ws,
                                             ws_bytes, s, flags, none);
  return run_scan_ops<float, CSR, false>(static_cast<const float *>(in), static_cast<float *>(out), a, ws, ws_bytes, s,
                                         flags, none);
}

}  // namespace desc
