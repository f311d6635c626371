// C-ABI entry points of the tgs library: argument validation, error reporting and dispatch to the
// kernel launchers. Every public function is declared in include/tgs.h.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "tgs_internal.cuh"

namespace tgs {

static thread_local char g_msg[512] = "";
static std::atomic<int64_t> g_launches{0};
static std::atomic<int64_t> g_allocations{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Every allocation of the library goes through these two (counted by tgs_allocation_count).
cudaError_t device_malloc(void** p, size_t bytes) {
  g_allocations.fetch_add(1, std::memory_order_relaxed);
  return cudaMalloc(p, bytes);
}
cudaError_t pinned_malloc(void** p, size_t bytes) {
  g_allocations.fetch_add(1, std::memory_order_relaxed);
  return cudaMallocHost(p, bytes);
}

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof g_msg, fmt, ap);
  va_end(ap);
}

tgs_status cuda_status(cudaError_t e, const char* what) {
  set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  return TGS_ERR_CUDA;
}

// The device-side error word: a zero-initialized int32 in this library's own device memory, one
// per device (a file-scope __device__ variable, so no call ever allocates it). Kernels receive its
// device address as an argument; the address is looked up once per device with
// cudaGetSymbolAddress and cached. The cache assumes the device's context lives as long as the
// process: after cudaDeviceReset the library must not be used again in that process.
static __device__ int32_t g_device_error = 0;

int32_t* device_error_word() {
  static std::mutex mu;
  static int32_t* words[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!words[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_error) != cudaSuccess) return nullptr;
    words[dev] = static_cast<int32_t*>(p);
  }
  return words[dev];
}

static bool valid_tiling(const tgs_tiling* t) {
  return t && t->group_w >= 1 && t->group_w <= TGS_MAX_GROUP && t->group_h >= 1 &&
         t->group_h <= TGS_MAX_GROUP && (t->flags & ~TGS_BIN_RANGE_ONLY) == 0;
}

static bool valid_size(int32_t w, int32_t h) { return w >= 1 && h >= 1 && w <= 16384 && h <= 16384; }

static int group_cols(int32_t w, const tgs_tiling* t) { return div_up(div_up(w, kTile), t->group_w); }
static int group_rows(int32_t h, const tgs_tiling* t) { return div_up(div_up(h, kTile), t->group_h); }

static tgs_status require_sm103(int32_t device) {
  cudaDeviceProp prop;
  TGS_CUDA(cudaGetDeviceProperties(&prop, device));
  if (prop.major != 10 || prop.minor != 3) {
    set_error("device %d is sm_%d%d; this library is built for sm_103a", device, prop.major,
              prop.minor);
    return TGS_ERR_UNSUPPORTED_DEVICE;
  }
  return TGS_OK;
}

static tgs_status require_current_sm103() {
  int dev = 0;
  TGS_CUDA(cudaGetDevice(&dev));
  static std::atomic<int> cached[64];  // 0 unknown, 1 ok, 2 unsupported (zero-initialized)
  if (dev >= 0 && dev < 64 && cached[dev].load(std::memory_order_relaxed) == 1) return TGS_OK;
  tgs_status s = require_sm103(dev);
  if (dev >= 0 && dev < 64) cached[dev].store((s == TGS_OK) ? 1 : 2, std::memory_order_relaxed);
  return s;
}

}  // namespace tgs

using namespace tgs;

extern "C" {

const char* tgs_status_string(tgs_status s) {
  switch (s) {
    case TGS_OK: return "TGS_OK";
    case TGS_ERR_INVALID_ARGUMENT: return "TGS_ERR_INVALID_ARGUMENT";
    case TGS_ERR_CUDA: return "TGS_ERR_CUDA";
    case TGS_ERR_CAPACITY: return "TGS_ERR_CAPACITY";
    case TGS_ERR_UNSUPPORTED_DEVICE: return "TGS_ERR_UNSUPPORTED_DEVICE";
    case TGS_ERR_TIMEOUT: return "TGS_ERR_TIMEOUT";
    case TGS_ERR_BUSY: return "TGS_ERR_BUSY";
    case TGS_ERR_NOT_FOUND: return "TGS_ERR_NOT_FOUND";
    default: return "TGS_ERR_UNKNOWN";
  }
}

const char* tgs_last_error_message(void) { return g_msg; }

int32_t tgs_abi_version(void) { return TGS_ABI_VERSION; }

int64_t tgs_kernel_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int64_t tgs_allocation_count(void) { return g_allocations.load(std::memory_order_relaxed); }

tgs_status tgs_check_device(int32_t device) { return require_sm103(device); }

tgs_status tgs_preprocess(const tgs_scene* scene, const tgs_camera* cam, tgs_projected* out,
                          void* stream) {
  g_msg[0] = 0;
  if (!scene || !cam || !out) return set_error("null argument"), TGS_ERR_INVALID_ARGUMENT;
  if (scene->n < 0 || scene->n >= (int64_t(1) << 31))
    return set_error("n = %lld out of range", (long long)scene->n), TGS_ERR_INVALID_ARGUMENT;
  if (scene->sh_degree < 0 || scene->sh_degree > 3)
    return set_error("sh_degree %d not in 0..3", scene->sh_degree), TGS_ERR_INVALID_ARGUMENT;
  if (!valid_size(cam->width, cam->height) || !(cam->fx > 0) || !(cam->fy > 0))
    return set_error("bad camera (size or focal length)"), TGS_ERR_INVALID_ARGUMENT;
  if (scene->n == 0) return TGS_OK;
  if (!scene->means || !scene->scales || !scene->quats || !scene->opacities || !scene->sh ||
      !out->mean2d || !out->conic_opacity || !out->rgb || !out->depth || !out->radius || !out->rect)
    return set_error("null array"), TGS_ERR_INVALID_ARGUMENT;
  tgs_status s = require_current_sm103();
  if (s != TGS_OK) return s;
  return launch_preprocess(*scene, *cam, *out, (cudaStream_t)stream);
}

tgs_status tgs_bin_sort_workspace_size(int64_t n, int64_t capacity, int32_t width, int32_t height,
                                       const tgs_tiling* tiling, size_t* bytes) {
  g_msg[0] = 0;
  if (!bytes || !valid_tiling(tiling) || !valid_size(width, height) || n < 0 || capacity < 0 ||
      capacity >= (int64_t(1) << 30) || n >= (int64_t(1) << 30))
    return set_error("bad argument"), TGS_ERR_INVALID_ARGUMENT;
  *bytes = bin_sort_workspace_bytes(n, capacity, group_cols(width, tiling), group_rows(height, tiling));
  return TGS_OK;
}

tgs_status tgs_bin_sort(const tgs_projected* proj, int64_t n, int32_t width, int32_t height,
                        const tgs_tiling* tiling, void* workspace, size_t workspace_bytes,
                        tgs_bins* bins, int64_t* num_entries_host, void* stream) {
  g_msg[0] = 0;
  if (!proj || !bins || !valid_tiling(tiling) || !valid_size(width, height) || n < 0 ||
      n >= (int64_t(1) << 30))
    return set_error("bad argument"), TGS_ERR_INVALID_ARGUMENT;
  if (bins->capacity < 0 || bins->capacity >= (int64_t(1) << 30))
    return set_error("capacity out of range"), TGS_ERR_INVALID_ARGUMENT;
  if (!bins->ranges || !bins->num_entries || (bins->capacity > 0 && (!bins->vals || !bins->masks)))
    return set_error("null bins array"), TGS_ERR_INVALID_ARGUMENT;
  if (n > 0 && (!proj->rect || !proj->depth || !proj->radius))
    return set_error("null projected array"), TGS_ERR_INVALID_ARGUMENT;
  const size_t need = bin_sort_workspace_bytes(n, bins->capacity, group_cols(width, tiling),
                                               group_rows(height, tiling));
  if (workspace_bytes < need || (need > 0 && !workspace) || ((uintptr_t)workspace & 255))
    return set_error("workspace too small or misaligned: need %zu bytes", need),
           TGS_ERR_INVALID_ARGUMENT;
  tgs_status s = require_current_sm103();
  if (s != TGS_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  s = launch_bin_sort(*proj, n, width, height, tiling->group_w, tiling->group_h,
                      (tiling->flags & TGS_BIN_RANGE_ONLY) == 0, workspace, workspace_bytes, *bins,
                      st);
  if (s != TGS_OK || !num_entries_host) return s;
  TGS_CUDA(cudaMemcpyAsync(num_entries_host, bins->num_entries, sizeof(int64_t),
                           cudaMemcpyDeviceToHost, st));
  int32_t failed = 0;
  if (n > 0)
    TGS_CUDA(cudaMemcpyAsync(&failed,
                             bin_sort_failed_word(workspace, n, bins->capacity,
                                                  group_cols(width, tiling), group_rows(height, tiling)),
                             sizeof failed, cudaMemcpyDeviceToHost, st));
  TGS_CUDA(cudaStreamSynchronize(st));
  if (failed) {
    set_error("a look-back wait of the bin sort ran out: the bins are empty");
    return TGS_ERR_TIMEOUT;
  }
  if (*num_entries_host > bins->capacity) {
    set_error("frame needs %lld entries, capacity %lld", (long long)*num_entries_host,
              (long long)bins->capacity);
    return TGS_ERR_CAPACITY;
  }
  return TGS_OK;
}

static tgs_status check_raster_args(const tgs_projected* proj, int64_t n, const tgs_bins* bins,
                                    int32_t width, int32_t height, const tgs_tiling* tiling,
                                    const tgs_raster_opts* opts) {
  if (!proj || !bins || !opts || !valid_tiling(tiling) || !valid_size(width, height) || n < 0 ||
      n >= (int64_t(1) << 31))
    return set_error("bad argument"), TGS_ERR_INVALID_ARGUMENT;
  if (!bins->ranges || (bins->capacity > 0 && (!bins->vals || !bins->masks)))
    return set_error("null bins array"), TGS_ERR_INVALID_ARGUMENT;
  if (n > 0 && (!proj->mean2d || !proj->conic_opacity || !proj->rgb))
    return set_error("null projected array"), TGS_ERR_INVALID_ARGUMENT;
  return TGS_OK;
}

tgs_status tgs_rasterize(const tgs_projected* proj, int64_t n, const tgs_bins* bins, int32_t width,
                         int32_t height, const tgs_tiling* tiling, const tgs_raster_opts* opts,
                         float* out_rgb, float* out_T, int32_t* n_contrib, void* stream) {
  g_msg[0] = 0;
  tgs_status s = check_raster_args(proj, n, bins, width, height, tiling, opts);
  if (s != TGS_OK) return s;
  if (!out_rgb || !out_T) return set_error("null output"), TGS_ERR_INVALID_ARGUMENT;
  s = require_current_sm103();
  if (s != TGS_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  switch (opts->precision) {
    case TGS_PRECISION_FP32:
      return launch_raster_fp32(*proj, *bins, width, height, tiling->group_w, tiling->group_h,
                                *opts, out_rgb, out_T, n_contrib, st);
    case TGS_PRECISION_FP16_TC:
    case TGS_PRECISION_BF16_TC:
      return launch_raster_tc(*proj, *bins, width, height, tiling->group_w, tiling->group_h, *opts,
                              out_rgb, out_T, n_contrib, st);
    default:
      set_error("unknown precision %d", opts->precision);
      return TGS_ERR_INVALID_ARGUMENT;
  }
}

tgs_status tgs_rasterize_batch(const tgs_frame* frames, int32_t count, const tgs_tiling* tiling,
                               const tgs_raster_opts* opts, int64_t wait_limit_ns, void* workspace,
                               void* stream) {
  g_msg[0] = 0;
  if (!frames || !opts || !valid_tiling(tiling) || count < 1 || count > TGS_BATCH_MAX_FRAMES)
    return set_error("bad argument (count %d, 1..%d frames)", count, TGS_BATCH_MAX_FRAMES),
           TGS_ERR_INVALID_ARGUMENT;
  if (opts->precision != TGS_PRECISION_FP16_TC && opts->precision != TGS_PRECISION_BF16_TC)
    return set_error("batched rasterization runs on the tensor cores (precision %d)", opts->precision),
           TGS_ERR_INVALID_ARGUMENT;
  if (opts->counters) return set_error("batched rasterization collects no counters"), TGS_ERR_INVALID_ARGUMENT;
  if (!workspace || ((uintptr_t)workspace & 3))
    return set_error("workspace of TGS_BATCH_WORKSPACE_BYTES device bytes needed"), TGS_ERR_INVALID_ARGUMENT;
  RasterFrame rf[TGS_BATCH_MAX_FRAMES];
  for (int f = 0; f < count; ++f) {
    const tgs_frame& fr = frames[f];
    const tgs_status s = check_raster_args(fr.proj, fr.n, fr.bins, fr.width, fr.height, tiling, opts);
    if (s != TGS_OK) {
      char m[512];
      snprintf(m, sizeof m, "%s", g_msg);
      return set_error("frame %d: %s", f, m), s;
    }
    if (!fr.out_rgb || !fr.out_T) return set_error("frame %d: null output", f), TGS_ERR_INVALID_ARGUMENT;
    rf[f] = RasterFrame{fr.proj, fr.bins, fr.width, fr.height, fr.out_rgb, fr.out_T, fr.ready,
                        fr.ready_value, fr.status, fr.done, fr.done_value};
  }
  tgs_status s = require_current_sm103();
  if (s != TGS_OK) return s;
  const uint64_t wait_ns = wait_limit_ns > 0 ? (uint64_t)wait_limit_ns : 2000000000ull;
  return launch_raster_tc_batch(rf, count, tiling->group_w, tiling->group_h, *opts,
                                static_cast<int*>(workspace), wait_ns, (cudaStream_t)stream);
}

tgs_status tgs_rasterize_backward(const tgs_projected* proj, int64_t n, const tgs_bins* bins,
                                  int32_t width, int32_t height, const tgs_tiling* tiling,
                                  const tgs_raster_opts* opts, const float* out_T,
                                  const int32_t* n_contrib, const float* grad_rgb,
                                  float* g_mean2d, float* g_conic_opacity, float* g_rgb,
                                  void* stream) {
  g_msg[0] = 0;
  tgs_status s = check_raster_args(proj, n, bins, width, height, tiling, opts);
  if (s != TGS_OK) return s;
  // the backward replays the FP32 forward's decisions: outputs of another precision's forward
  // would give the gradient of a different image
  if (opts->precision != TGS_PRECISION_FP32)
    return set_error("the backward needs the outputs of an FP32 forward (precision %d given)",
                     opts->precision),
           TGS_ERR_INVALID_ARGUMENT;
  if (!out_T || !n_contrib || !grad_rgb || (n > 0 && (!g_mean2d || !g_conic_opacity || !g_rgb)))
    return set_error("null argument"), TGS_ERR_INVALID_ARGUMENT;
  s = require_current_sm103();
  if (s != TGS_OK) return s;
  return launch_raster_backward(*proj, n, *bins, width, height, tiling->group_w, tiling->group_h,
                                *opts, out_T, n_contrib, grad_rgb, g_mean2d, g_conic_opacity, g_rgb,
                                (cudaStream_t)stream);
}

int64_t tgs_set_lookback_limit(int64_t ns) { return set_lookback_limit_ns(ns); }

tgs_status tgs_last_device_error(int32_t reset) {
  g_msg[0] = 0;
  int32_t* w = device_error_word();
  if (!w) return set_error("device error word unavailable"), TGS_ERR_CUDA;
  TGS_CUDA(cudaDeviceSynchronize());
  int32_t v = 0;
  TGS_CUDA(cudaMemcpy(&v, w, sizeof v, cudaMemcpyDeviceToHost));
  if (reset) TGS_CUDA(cudaMemset(w, 0, sizeof(int32_t)));
  if (v != TGS_OK) set_error("a device pipeline wait expired (code %d)", v);
  return v;
}

}  // extern "C"
