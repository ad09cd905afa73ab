// Scans through lowered maps of two canonical dims (the columns of a
// matrix, a reversed row order, ...): the look-back scan of k_scan_core.cuh
// with each address decoded from the map, in a translation unit of its own
// so that the build compiles it beside the one-dim forms.
#include "k_scan_core.cuh"

namespace desc {

int32_t scan_status_take_mapped2() { return take_status_word(); }

int32_t launch_scan_mapped_2d(int32_t dtype, const void *in, void *out, int64_t off, const int64_t *ext,
                              const int64_t *stride, int nd, int64_t period, int32_t flags, void *ws,
                              size_t ws_bytes, desc_stream_t st) {
  if (flags & kMapScanOps) return DESC_ERR_INVALID_ARG;
  MapArgs m;
  const int64_t n = build_map(off, ext, stride, nd, period, &m);
  if (n == 0) return DESC_OK;
  if (m.nd != 2 || !m.fast) return DESC_ERR_INVALID_ARG;   // launch_scan_mapped routes only these here
  return run_scan_mapped_nd<2>(dtype, in, out, m, n, period, flags, ws, ws_bytes, reinterpret_cast<cudaStream_t>(st));
}

}  // namespace desc
