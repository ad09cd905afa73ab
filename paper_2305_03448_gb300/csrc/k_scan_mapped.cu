// Scans of views whose lowered map is not one contiguous run, through the
// look-back scan of k_scan_core.cuh with every address taken from the map
// (maps of up to two canonical dims; others go to the one-tile map scan).
#include "k_scan_core.cuh"

namespace desc {

int32_t scan_status_take_mapped() { return take_status_word(); }

int32_t launch_scan_mapped(int32_t dtype, const void *in, void *out, int64_t off, const int64_t *ext,
                           const int64_t *stride, int nd, int64_t period, int32_t flags, void *ws, size_t ws_bytes,
                           desc_stream_t st) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  if (flags & kMapScanOps) return DESC_ERR_INVALID_ARG;   // arg operators: launch_scan_map
  MapArgs m;
  const int64_t n = build_map(off, ext, stride, nd, period, &m);
  if (n == 0) return DESC_OK;
  if (m.nd > 2 || !m.fast)                             // the one-tile map scan decodes any map
    return launch_scan_map(dtype, in, out, off, ext, stride, nd, period, nullptr, 0, nullptr, flags, ws, ws_bytes,
                           st);
  ScanArgs a{};
  a.n = n;
  a.period = period > 0 ? period : n;
  a.debug = (flags & DESC_DEBUG_STALL_TILE) ? 1 : 0;
  a.vec = map_vec(m, in, out) ? 1 : 0;
  const bool periodic = a.period < n;
  const bool basic = !(flags & (DESC_PROD | DESC_AND | DESC_OR | DESC_XOR));
  auto go = [&](auto tag) -> int32_t {
    using T = decltype(tag);
    auto i = static_cast<const T *>(in);
    auto o = static_cast<T *>(out);
    if (basic)
      return periodic ? run_scan_basic<T, PERIODIC, true>(i, o, a, ws, ws_bytes, s, -1, flags, m)
                      : run_scan_basic<T, PLAIN, true>(i, o, a, ws, ws_bytes, s, -1, flags, m);
    return periodic ? run_scan_ops<T, PERIODIC, true>(i, o, a, ws, ws_bytes, s, flags, m)
                    : run_scan_ops<T, PLAIN, true>(i, o, a, ws, ws_bytes, s, flags, m);
  };
  return dtype == DESC_I32 ? go(int32_t(0)) : go(0.f);
}

}  // namespace desc
