// Fixed scratch for desc_scan_noalloc: a scan that allocates nothing.
//
// The look-back scan needs a small scratch area (a tile ticket, an abort
// flag and one status pair per tile).  Here that scratch is a file-scope
// device array, so the caller passes only its input and output buffers.
// Every GPU that loads the library holds the array until the process exits.
//
// Host code cannot use the array's name as a device address (in host code
// it names a host-side stand-in), so the address is looked up with
// cudaGetSymbolAddress once per device, with that device current, and
// passed to the kernel like any other workspace pointer.
#include <cuda_runtime.h>

#include <mutex>

#include "desc_internal.h"

namespace desc {
namespace {

// 256 bytes of header (ticket, abort flag) + one tile state per tile of
// kScanNoallocTile elements.
constexpr size_t kNoallocScratchBytes =
    256 + size_t(DESC_SCAN_NOALLOC_MAX_ELEMS / kScanNoallocTile) * kScanTileStateBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up on the
// first call for that device).
int32_t scratch_for_current_device(void **ptr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DESC_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return DESC_ERR_CUDA;
    }
    g_ptr[dev] = p;
  }
  *ptr = g_ptr[dev];
  return DESC_OK;
}

}  // namespace

int32_t launch_scan_contig_noalloc(int32_t dtype, const void *in, void *out, int64_t n,
                                   int64_t period, desc_stream_t s) {
  if (n > DESC_SCAN_NOALLOC_MAX_ELEMS) return DESC_ERR_WORKSPACE;
  void *ws = nullptr;
  const int32_t r = scratch_for_current_device(&ws);
  if (r != DESC_OK) return r;
  return launch_scan_contig(dtype, in, out, n, period, 0, ws, kNoallocScratchBytes, s, -1);
}

}  // namespace desc
