// Scans of views whose lowered map is not one contiguous run, through the
// look-back scan of k_scan_core.cuh with every address taken from the map:
// maps of one canonical dim here, two in k_scan_mapped2.cu, others in the
// one-tile map scan.
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
  if (m.nd == 2 && m.fast)
    return launch_scan_mapped_2d(dtype, in, out, off, ext, stride, nd, period, flags, ws, ws_bytes, st);
  if (m.nd == 0) {                                     // off + g
    m.nd = 1;
    m.ext[0] = n;
    m.st[0] = 1;
  }
  const int64_t lim = int64_t(1) << 31;
  if (m.nd != 1 || n >= lim || m.st[0] >= lim || m.st[0] <= -lim)   // the one-tile map scan decodes any map
    return launch_scan_map(dtype, in, out, off, ext, stride, nd, period, nullptr, 0, nullptr, flags, ws, ws_bytes,
                           st);
  return run_scan_mapped_nd<1>(dtype, in, out, m, n, period, flags, ws, ws_bytes, s);
}

}  // namespace desc
