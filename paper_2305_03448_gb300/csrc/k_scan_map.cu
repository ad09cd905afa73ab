// The one-tile map scan (any lowered map, every operator; the arg operators
// run only here) and the per-segment group schedules of the CSR call, from
// k_scan_core.cuh.
#include <mutex>
#include <set>
#include <utility>

#include "k_scan_core.cuh"

namespace desc {

int32_t scan_status_take_map() { return take_status_word(); }

int32_t launch_scan_map(int32_t dtype, const void *in, void *out, int64_t off, const int64_t *ext,
                        const int64_t *stride, int nd, int64_t period, const int64_t *offsets, int64_t nseg,
                        void *sums, int32_t flags, void *ws, size_t ws_bytes, desc_stream_t st) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  MapArgs m;
  const int64_t n = build_map(off, ext, stride, nd, period, &m);
  if (n == 0) return DESC_OK;
  const int64_t ntiles = (n + kMapTile - 1) / kMapTile;
  const size_t need = align256(sizeof(ScanWs)) + size_t(ntiles) * sizeof(TileState);
  if (!ws || ws_bytes < need) return DESC_ERR_WORKSPACE;
  if (ntiles >= (int64_t(1) << 31)) return DESC_ERR_UNSUPPORTED;
  ScanArgs a{};
  a.n = n;
  a.period = period > 0 ? period : n;
  a.offsets = offsets;
  a.nseg = nseg;
  a.sums = sums;
  a.debug = (flags & DESC_DEBUG_STALL_TILE) ? 1 : 0;
  a.vec = map_vec(m, in, out) ? 1 : 0;
  const int mode = offsets ? CSR : (a.period < n ? PERIODIC : PLAIN);
  const int excl = (flags & DESC_EXCLUSIVE) ? 1 : 0;
  DESC_CUDA_TRY(cudaMemsetAsync(ws, 0, need, s));
  ScanWs *w = static_cast<ScanWs *>(ws);
  TileState *ts = reinterpret_cast<TileState *>(static_cast<char *>(ws) + align256(sizeof(ScanWs)));
  return with_states(dtype, flags, [&](auto tag) {
    using T = typename decltype(tag)::Elem;
    using S = typename decltype(tag)::States;
    scan_map_kernel<T, S><<<(unsigned)ntiles, kMapThreads + 32, 0, s>>>(static_cast<const T *>(in),
                                                                         static_cast<uint32_t *>(out), m, a, w, ts,
                                                                         mode, excl);
    DESC_CUDA_TRY(cudaGetLastError());
    return DESC_OK;
  });
}

namespace {
// The arg kernels' shared memory (above the default 48 KB) is allowed once
// per kernel and device.
cudaError_t allow_arg_smem(const void *kernel) {
  static std::mutex mu;
  static std::set<std::pair<const void *, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({kernel, dev})) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kArgSmem);
  if (e == cudaSuccess) done.insert({kernel, dev});
  return e;
}
}  // namespace

int32_t launch_scan_arg(int32_t dtype, const void *in, void *out, int64_t n, int64_t period, const int64_t *offsets,
                        int64_t nseg, void *sums, int64_t idx_base, int32_t flags, void *ws, size_t ws_bytes,
                        desc_stream_t st) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  const int64_t ntiles = (n + kArgTile - 1) / kArgTile;
  if (ntiles == 0) return DESC_OK;
  const size_t need = align256(sizeof(ScanWs)) + size_t(ntiles) * sizeof(TileState);
  if (!ws || ws_bytes < need) return DESC_ERR_WORKSPACE;
  if (ntiles >= (int64_t(1) << 31)) return DESC_ERR_UNSUPPORTED;
  ScanArgs a{};
  a.n = n;
  a.period = period > 0 ? period : n;
  a.offsets = offsets;
  a.nseg = nseg;
  a.sums = sums;
  a.debug = (flags & DESC_DEBUG_STALL_TILE) ? 1 : 0;
  a.vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
  const int mode = offsets ? CSR : (a.period < n ? PERIODIC : PLAIN);
  const bool mx = (flags & DESC_ARGMAX) != 0, ex = (flags & DESC_EXCLUSIVE) != 0;
  DESC_CUDA_TRY(cudaMemsetAsync(ws, 0, need, s));
  ScanWs *w = static_cast<ScanWs *>(ws);
  TileState *ts = reinterpret_cast<TileState *>(static_cast<char *>(ws) + align256(sizeof(ScanWs)));
  auto launch = [&](auto kernel, auto typed_in) -> int32_t {
    DESC_CUDA_TRY(allow_arg_smem(reinterpret_cast<const void *>(kernel)));
    kernel<<<(unsigned)ntiles, kThreads + 32, kArgSmem, s>>>(typed_in, static_cast<int32_t *>(out), with_period(a),
                                                              idx_base, w, ts, MapArgs{});
    DESC_CUDA_TRY(cudaGetLastError());
    return DESC_OK;
  };
  auto with_mode = [&](auto tag, auto maxv) -> int32_t {
    using T = decltype(tag);
    constexpr bool MX = decltype(maxv)::value;
    const T *ti = static_cast<const T *>(in);
    if (mode == CSR)
      return ex ? launch(scan_arg_kernel<T, MX, CSR, true>, ti) : launch(scan_arg_kernel<T, MX, CSR, false>, ti);
    if (mode == PERIODIC)
      return ex ? launch(scan_arg_kernel<T, MX, PERIODIC, true>, ti)
                : launch(scan_arg_kernel<T, MX, PERIODIC, false>, ti);
    return ex ? launch(scan_arg_kernel<T, MX, PLAIN, true>, ti) : launch(scan_arg_kernel<T, MX, PLAIN, false>, ti);
  };
  if (dtype == DESC_I32)
    return mx ? with_mode(int32_t(0), std::true_type{}) : with_mode(int32_t(0), std::false_type{});
  return mx ? with_mode(0.f, std::true_type{}) : with_mode(0.f, std::false_type{});
}

int32_t launch_seg_group(int32_t dtype, const void *in, void *out, const int64_t *offsets, int64_t nseg, void *sums,
                         int32_t flags, int threads, desc_stream_t st) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  const bool ex = (flags & DESC_EXCLUSIVE) != 0;
  auto go = [&](auto tag) -> int32_t {
    using T = decltype(tag);
    const T *i = static_cast<const T *>(in);
    T *o = static_cast<T *>(out);
    T *sm = static_cast<T *>(sums);
    if (flags & DESC_MAX)
      return ex ? run_seg_group<T, ExtOp<T, true>, true>(i, o, offsets, nseg, sm, threads, s)
                : run_seg_group<T, ExtOp<T, true>, false>(i, o, offsets, nseg, sm, threads, s);
    if (flags & DESC_MIN)
      return ex ? run_seg_group<T, ExtOp<T, false>, true>(i, o, offsets, nseg, sm, threads, s)
                : run_seg_group<T, ExtOp<T, false>, false>(i, o, offsets, nseg, sm, threads, s);
    return ex ? run_seg_group<T, SumOp<T>, true>(i, o, offsets, nseg, sm, threads, s)
              : run_seg_group<T, SumOp<T>, false>(i, o, offsets, nseg, sm, threads, s);
  };
  return dtype == DESC_I32 ? go(int32_t(0)) : go(0.f);
}

}  // namespace desc
