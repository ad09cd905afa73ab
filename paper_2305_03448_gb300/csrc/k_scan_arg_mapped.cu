// Arg-maximum / arg-minimum scans through lowered maps of one or two
// canonical dims (a reversed array, the columns of a matrix, ...): the arg
// look-back scan of k_scan_core.cuh with each point's element index taken
// from the map.  Maps it cannot decode go to the one-tile map scan.
#include "k_scan_core.cuh"

namespace desc {

static_assert(kArgSmem <= 48 * 1024, "the mapped arg scan launches within the default shared-memory limit");

int32_t scan_status_take_argmap() { return take_status_word(); }

namespace {

template <int ND>
int32_t run_arg_mapped(int32_t dtype, const void *in, void *out, const MapArgs &m, int64_t n, int64_t period,
                       int32_t flags, void *ws, size_t ws_bytes, cudaStream_t s) {
  const int64_t ntiles = (n + kArgTile - 1) / kArgTile;
  const size_t need = align256(sizeof(ScanWs)) + size_t(ntiles) * sizeof(TileState);
  if (!ws || ws_bytes < need) return DESC_ERR_WORKSPACE;
  if (ntiles >= (int64_t(1) << 31)) return DESC_ERR_UNSUPPORTED;
  ScanArgs a{};
  a.n = n;
  a.period = period > 0 ? period : n;
  a.debug = (flags & DESC_DEBUG_STALL_TILE) ? 1 : 0;
  a.vec = map_load_mode(m, in, out);
  const bool periodic = a.period < n;
  const bool mx = (flags & DESC_ARGMAX) != 0, ex = (flags & DESC_EXCLUSIVE) != 0;
  DESC_CUDA_TRY(cudaMemsetAsync(ws, 0, need, s));
  ScanWs *w = static_cast<ScanWs *>(ws);
  TileState *ts = reinterpret_cast<TileState *>(static_cast<char *>(ws) + align256(sizeof(ScanWs)));
  auto launch = [&](auto kernel, auto typed_in) -> int32_t {
    kernel<<<(unsigned)ntiles, kThreads + 32, kArgSmem, s>>>(typed_in, static_cast<int32_t *>(out), with_period(a),
                                                              0, w, ts, m);
    DESC_CUDA_TRY(cudaGetLastError());
    return DESC_OK;
  };
  auto with_mode = [&](auto tag, auto maxv) -> int32_t {
    using T = decltype(tag);
    constexpr bool MX = decltype(maxv)::value;
    constexpr int P3 = 3, P4 = kArgBlocksPerSM;
    const T *ti = static_cast<const T *>(in);
    if (periodic)
      return ex ? launch(scan_arg_kernel<T, MX, PERIODIC, true, kArgSub, kArgPipe, P3, ND>, ti)
                : launch(scan_arg_kernel<T, MX, PERIODIC, false, kArgSub, kArgPipe, P3, ND>, ti);
    return ex ? launch(scan_arg_kernel<T, MX, PLAIN, true, kArgSub, kArgPipe, P4, ND>, ti)
              : launch(scan_arg_kernel<T, MX, PLAIN, false, kArgSub, kArgPipe, P4, ND>, ti);
  };
  auto with_op = [&](auto tag) -> int32_t {
    return mx ? with_mode(tag, std::true_type{}) : with_mode(tag, std::false_type{});
  };
  return dtype == DESC_I32 ? with_op(int32_t(0)) : with_op(0.f);
}

}  // namespace

int32_t launch_scan_arg_mapped(int32_t dtype, const void *in, void *out, int64_t off, const int64_t *ext,
                               const int64_t *stride, int nd, int64_t period, int32_t flags, void *ws,
                               size_t ws_bytes, desc_stream_t st) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  if (!(flags & kArgFlags)) return DESC_ERR_INVALID_ARG;
  MapArgs m;
  const int64_t n = build_map(off, ext, stride, nd, period, &m);
  if (n == 0) return DESC_OK;
  if (m.nd == 0) {                                     // off + g
    m.nd = 1;
    m.ext[0] = n;
    m.st[0] = 1;
  }
  const int64_t lim = int64_t(1) << 31;
  if (m.nd == 1 && n < lim && m.st[0] < lim && m.st[0] > -lim)
    return run_arg_mapped<1>(dtype, in, out, m, n, period, flags, ws, ws_bytes, s);
  if (m.nd == 2 && m.fast) return run_arg_mapped<2>(dtype, in, out, m, n, period, flags, ws, ws_bytes, s);
  return launch_scan_map(dtype, in, out, off, ext, stride, nd, period, nullptr, 0, nullptr, flags, ws, ws_bytes, st);
}

}  // namespace desc
