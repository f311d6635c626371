// tgs_bin_sort_static: the bin sort for callers that cannot allocate device memory.
//
// Some callers of this library must not allocate device memory once they are running: a real-time
// frame loop or a VR compositor that fixes its memory budget at start-up, or a host application
// that owns every device allocation and hands plugins no allocator. tgs_bin_sort needs a scratch
// workspace from its caller; this entry point instead uses a fixed scratch area that lives inside
// the library as a file-scope __device__ array. Every GPU that loads the library holds that area
// until the process exits, so its size is kept modest (TGS_BIN_SORT_STATIC_BYTES).
//
// It allocates nothing, on its first call as on every other: no cudaMalloc, cudaFree or allocating
// library call (the library's device error word is a __device__ variable too). On its first call
// on a device (with that device current) it looks up the device address of the array with
// cudaGetSymbolAddress and caches it. CUDA loads a library's device code lazily, so that first
// call is also when the array's memory is committed on the device: a caller with a memory budget
// fixed at start-up should make it then, before any stream capture. All calls share the one array
// and it keeps the last call's contents; the bin sort writes every scratch word it reads (and
// clears its counters itself), so nothing needs clearing, but calls whose work overlaps on the GPU
// (different streams, or different host threads on the same device) race on the array.
#include <mutex>

#include "tgs_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = TGS_BIN_SORT_STATIC_BYTES;

// The scratch area. In host code this name is only a host-side stand-in for the symbol: it is
// never passed to a kernel; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_bin_sort_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_scratch[64] = {nullptr};  // per-device address of g_bin_sort_scratch

tgs_status scratch_address(void** out) {
  int dev = 0;
  TGS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    tgs::set_error("device index %d out of range", dev);
    return TGS_ERR_INVALID_ARGUMENT;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_bin_sort_scratch);
    if (e == cudaErrorMemoryAllocation) {
      tgs::set_error("loading the %zu-byte static bin-sort scratch on device %d failed: out of "
                     "device memory (make the first tgs_bin_sort_static call at start-up)",
                     kStaticScratchBytes, dev);
      return TGS_ERR_CUDA;
    }
    if (e != cudaSuccess) return tgs::cuda_status(e, "cudaGetSymbolAddress(bin sort scratch)");
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return TGS_OK;
}

}  // namespace

extern "C" tgs_status tgs_bin_sort_static(const tgs_projected* proj, int64_t n, int32_t width,
                                          int32_t height, const tgs_tiling* tiling, tgs_bins* bins,
                                          int64_t* num_entries_host, void* stream) {
  if (!bins) {
    tgs::set_error("null bins");
    return TGS_ERR_INVALID_ARGUMENT;
  }
  size_t need = 0;
  tgs_status s = tgs_bin_sort_workspace_size(n, bins->capacity, width, height, tiling, &need);
  if (s != TGS_OK) return s;
  if (need > kStaticScratchBytes) {
    tgs::set_error(
        "tgs_bin_sort_static: %lld Gaussians with capacity %lld need %zu bytes of scratch; the "
        "static area holds %zu bytes (use tgs_bin_sort with a caller workspace)",
        (long long)n, (long long)bins->capacity, need, kStaticScratchBytes);
    if (num_entries_host) *num_entries_host = -1;  // not a frame's entry count
    return TGS_ERR_CAPACITY;
  }
  void* ws = nullptr;
  s = scratch_address(&ws);
  if (s != TGS_OK) return s;
  return tgs_bin_sort(proj, n, width, height, tiling, ws, kStaticScratchBytes, bins,
                      num_entries_host, stream);
}
