// Frame sequences from host memory (tgs_frames_*): the Section 2 pipeline (preprocess -> bin sort
// -> rasterize, Algorithm 1) per camera, fed from a scene in host memory and writing host images,
// with the copies overlapped with the kernels.
//
// Streams and buffers of one object:
//   upload stream      copies a call's scene into device copy (call % 2), after the frames of the
//                      call two back (the previous user of that copy) have finished reading it;
//   prep stream s      (one per buffer set, highest priority) preprocess + bin sort of the frames
//                      that take set s, after the scene copy is in and set s's previous image has
//                      been downloaded;
//   raster stream      every rasterization, in frame order, each after its set's bin sort;
//   download stream    every image (and T) copy to the host, each after its rasterization.
// So the next call's upload, the bin sorts of the next frames, the current rasterization and the
// previous frames' downloads all run at once. Nothing is allocated after tgs_frames_create.
#include <algorithm>
#include <vector>

#include "groupings.h"
#include "tgs_internal.cuh"

namespace tgs {
namespace {

constexpr int kMaxSets = 8;

inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct SceneCopy {
  float *means = nullptr, *scales = nullptr, *quats = nullptr, *opac = nullptr, *sh = nullptr;
};

struct FrameSet {
  tgs_projected proj{};
  tgs_bins bins{};
  void* ws = nullptr;
  size_t ws_bytes = 0;
  float* rgb = nullptr;  // [3, H, W] of the frame's size
  float* T = nullptr;    // [H, W]
  cudaStream_t prep = nullptr;
  cudaEvent_t prepped = nullptr;  // preprocess + bin sort done
  cudaEvent_t drawn = nullptr;    // rasterization done
  cudaEvent_t free = nullptr;     // image downloaded: the set may be reused
  bool used = false;
};

}  // namespace
}  // namespace tgs

struct tgs_frames {
  tgs_frames_config cfg{};
  int device = 0;
  void* mem = nullptr;  // one device block for every buffer
  size_t bytes = 0;
  int32_t* words = nullptr;  // device [0] bin-sort time-out, [1] capacity overflow
  tgs::SceneCopy scene[2];
  cudaEvent_t scene_in[2] = {nullptr, nullptr};    // upload into copy b complete
  cudaEvent_t scene_free[2] = {nullptr, nullptr};  // frames that read copy b complete
  bool scene_used[2] = {false, false};
  std::vector<tgs::FrameSet> sets;
  cudaStream_t upload = nullptr, raster = nullptr, download = nullptr;
  cudaEvent_t done = nullptr;  // last download of the last call
  int64_t calls = 0, frames = 0;
};

namespace tgs {
namespace {

struct Guard {  // makes the object's device current for the duration of a call
  int prev = -1;
  cudaError_t status;
  explicit Guard(int dev) {
    cudaGetDevice(&prev);
    status = cudaSetDevice(dev);
  }
  ~Guard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int64_t groups_of(const tgs_frames_config& c, int* GX, int* GY) {
  *GX = div_up(div_up(c.max_width, kTile), c.tiling.group_w);
  *GY = div_up(div_up(c.max_height, kTile), c.tiling.group_h);
  return (int64_t)*GX * *GY;
}

// Bytes of all device buffers, and their addresses inside F->mem when `place` is set.
size_t layout(tgs_frames* F, bool place) {
  const tgs_frames_config& c = F->cfg;
  const int64_t n = c.max_gaussians, cap = c.max_entries;
  const int64_t shf = 3 * (int64_t)(c.max_sh_degree + 1) * (c.max_sh_degree + 1);
  int GX = 0, GY = 0;
  const int64_t G = groups_of(c, &GX, &GY);
  const size_t ws = bin_sort_workspace_bytes(n, cap, GX, GY);
  const size_t px = (size_t)c.max_width * c.max_height;
  char* base = place ? static_cast<char*>(F->mem) : nullptr;
  size_t off = 0;
  auto take = [&](size_t b) {
    char* q = base ? base + off : nullptr;
    off += al256(b);
    return q;
  };
  F->words = reinterpret_cast<int32_t*>(take(16));
  for (SceneCopy& s : F->scene) {
    s.means = reinterpret_cast<float*>(take(12 * n));
    s.scales = reinterpret_cast<float*>(take(12 * n));
    s.quats = reinterpret_cast<float*>(take(16 * n));
    s.opac = reinterpret_cast<float*>(take(4 * n));
    s.sh = reinterpret_cast<float*>(take(4 * shf * n));
  }
  for (FrameSet& f : F->sets) {
    f.proj.mean2d = reinterpret_cast<float*>(take(8 * n));
    f.proj.conic_opacity = reinterpret_cast<float*>(take(16 * n));
    f.proj.rgb = reinterpret_cast<float*>(take(12 * n));
    f.proj.depth = reinterpret_cast<float*>(take(4 * n));
    f.proj.radius = reinterpret_cast<int32_t*>(take(4 * n));
    f.proj.rect = reinterpret_cast<int32_t*>(take(16 * n));
    f.bins.capacity = cap;
    f.bins.keys = nullptr;
    f.bins.vals = reinterpret_cast<uint32_t*>(take(4 * cap));
    f.bins.masks = reinterpret_cast<uint16_t*>(take(2 * cap));
    f.bins.ranges = reinterpret_cast<uint32_t*>(take(8 * G));
    f.bins.num_entries = reinterpret_cast<int64_t*>(take(8));
    f.ws = take(ws);
    f.ws_bytes = ws;
    f.rgb = reinterpret_cast<float*>(take(12 * px));
    f.T = reinterpret_cast<float*>(take(4 * px));
  }
  return off;
}

void release(tgs_frames* F) {
  for (FrameSet& f : F->sets) {
    if (f.prep) cudaStreamDestroy(f.prep);
    if (f.prepped) cudaEventDestroy(f.prepped);
    if (f.drawn) cudaEventDestroy(f.drawn);
    if (f.free) cudaEventDestroy(f.free);
  }
  for (int b = 0; b < 2; ++b) {
    if (F->scene_in[b]) cudaEventDestroy(F->scene_in[b]);
    if (F->scene_free[b]) cudaEventDestroy(F->scene_free[b]);
  }
  if (F->upload) cudaStreamDestroy(F->upload);
  if (F->raster) cudaStreamDestroy(F->raster);
  if (F->download) cudaStreamDestroy(F->download);
  if (F->done) cudaEventDestroy(F->done);
  if (F->mem) cudaFree(F->mem);
  delete F;
}

bool valid_config(const tgs_frames_config& c) {
  return c.max_gaussians >= 1 && c.max_gaussians < (int64_t(1) << 30) && c.max_sh_degree >= 0 &&
         c.max_sh_degree <= 3 && c.max_width >= 1 && c.max_width <= 16384 && c.max_height >= 1 &&
         c.max_height <= 16384 && c.max_entries >= 1 && c.max_entries < (int64_t(1) << 30) &&
         (c.tiling.flags & ~TGS_BIN_RANGE_ONLY) == 0 &&
         (c.precision == TGS_PRECISION_FP32 || c.precision == TGS_PRECISION_FP16_TC ||
          c.precision == TGS_PRECISION_BF16_TC) &&
         grouping_supported(c.precision, c.tiling.group_w, c.tiling.group_h) &&
         c.sets >= 2 && c.sets <= kMaxSets;
}

}  // namespace
}  // namespace tgs

using namespace tgs;

extern "C" {

tgs_status tgs_frames_create(const tgs_frames_config* config, tgs_frames** out) {
  if (!config || !out) return set_error("null argument"), TGS_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  if (!valid_config(*config)) return set_error("bad frames config"), TGS_ERR_INVALID_ARGUMENT;
  tgs_status s = tgs_check_device(config->device);
  if (s != TGS_OK) return s;
  Guard guard(config->device);
  TGS_CUDA(guard.status);
  auto* F = new tgs_frames;
  F->cfg = *config;
  F->device = config->device;
  F->sets.resize(config->sets);
  F->bytes = layout(F, false);
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  auto fail = [&](cudaError_t e, const char* what) {
    release(F);
    return cuda_status(e, what);
  };
  cudaError_t e = device_malloc(&F->mem, F->bytes);
  if (e != cudaSuccess) return fail(e, "frames buffers");
  layout(F, true);
  const unsigned flags = cudaStreamNonBlocking;
  e = cudaStreamCreateWithPriority(&F->upload, flags, lo);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&F->raster, flags, lo);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&F->download, flags, lo);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&F->done, cudaEventDisableTiming);
  for (int b = 0; e == cudaSuccess && b < 2; ++b) {
    e = cudaEventCreateWithFlags(&F->scene_in[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&F->scene_free[b], cudaEventDisableTiming);
  }
  for (FrameSet& f : F->sets) {
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&f.prep, flags, hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f.prepped, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f.drawn, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f.free, cudaEventDisableTiming);
  }
  // the status words start at 0 (ordered before every later call by the upload stream's events)
  if (e == cudaSuccess) e = cudaMemsetAsync(F->words, 0, 16, F->upload);
  if (e == cudaSuccess) e = cudaStreamSynchronize(F->upload);
  if (e != cudaSuccess) return fail(e, "frames streams");
  *out = F;
  return TGS_OK;
}

int64_t tgs_frames_device_bytes(const tgs_frames* F) { return F ? (int64_t)F->bytes : 0; }

}  // extern "C"

extern "C" {

tgs_status tgs_frames_render(tgs_frames* F, const tgs_scene* scene, const tgs_camera* cams,
                             int32_t count, float* out_rgb, float* out_T, void* stream) {
  if (!F || !scene || count < 0 || (count > 0 && (!cams || !out_rgb)))
    return set_error("null argument or negative count"), TGS_ERR_INVALID_ARGUMENT;
  if (count == 0) return TGS_OK;
  const tgs_frames_config& c = F->cfg;
  const int64_t n = scene->n;
  if (n < 0 || n > c.max_gaussians || scene->sh_degree < 0 || scene->sh_degree > c.max_sh_degree)
    return set_error("scene of %lld Gaussians, SH degree %d: the object holds %lld, degree %d",
                     (long long)n, scene->sh_degree, (long long)c.max_gaussians, c.max_sh_degree),
           TGS_ERR_INVALID_ARGUMENT;
  if (n > 0 && (!scene->means || !scene->scales || !scene->quats || !scene->opacities || !scene->sh))
    return set_error("null scene array"), TGS_ERR_INVALID_ARGUMENT;
  const int W = cams[0].width, H = cams[0].height;
  for (int k = 0; k < count; ++k) {
    const tgs_camera& q = cams[k];
    if (q.width != W || q.height != H || q.fx <= 0.f || q.fy <= 0.f)
      return set_error("camera %d: cameras of one call share one size and need fx, fy > 0", k),
             TGS_ERR_INVALID_ARGUMENT;
  }
  if (W < 1 || H < 1 || W > c.max_width || H > c.max_height)
    return set_error("%dx%d frames: the object holds %dx%d", W, H, c.max_width, c.max_height),
           TGS_ERR_INVALID_ARGUMENT;
  Guard guard(F->device);
  TGS_CUDA(guard.status);
  // upload into the scene copy the previous call did not use, once the frames that last read it
  // are done
  const int b = (int)(F->calls % 2);
  const SceneCopy& d = F->scene[b];
  if (F->scene_used[b]) TGS_CUDA(cudaStreamWaitEvent(F->upload, F->scene_free[b], 0));
  if (n > 0) {
    const size_t shf = 3 * (size_t)(scene->sh_degree + 1) * (scene->sh_degree + 1);
    const cudaMemcpyKind h2d = cudaMemcpyHostToDevice;
    TGS_CUDA(cudaMemcpyAsync(d.means, scene->means, 12 * (size_t)n, h2d, F->upload));
    TGS_CUDA(cudaMemcpyAsync(d.scales, scene->scales, 12 * (size_t)n, h2d, F->upload));
    TGS_CUDA(cudaMemcpyAsync(d.quats, scene->quats, 16 * (size_t)n, h2d, F->upload));
    TGS_CUDA(cudaMemcpyAsync(d.opac, scene->opacities, 4 * (size_t)n, h2d, F->upload));
    TGS_CUDA(cudaMemcpyAsync(d.sh, scene->sh, 4 * shf * (size_t)n, h2d, F->upload));
  }
  TGS_CUDA(cudaEventRecord(F->scene_in[b], F->upload));
  const tgs_scene ds{n, scene->sh_degree, d.means, d.scales, d.quats, d.opac, d.sh};
  tgs_raster_opts o{};
  o.precision = c.precision;
  for (int k = 0; k < 3; ++k) o.bg[k] = c.bg[k];
  const bool membership = (c.tiling.flags & TGS_BIN_RANGE_ONLY) == 0;
  const int gw = c.tiling.group_w, gh = c.tiling.group_h;
  const size_t px = (size_t)W * H;
  // A launch that fails stops the call, but the frame's events are still recorded and the call is
  // closed as a complete one would be, so the next call waits for whatever this one enqueued.
  tgs_status s = TGS_OK;
  for (int k = 0; k < count && s == TGS_OK; ++k) {
    FrameSet& f = F->sets[F->frames % (int64_t)F->sets.size()];
    ++F->frames;
    // preprocess + bin sort once the scene is in and the set's previous image has been copied out
    // (which follows the rasterization that read the set's bins)
    TGS_CUDA(cudaStreamWaitEvent(f.prep, F->scene_in[b], 0));
    if (f.used) TGS_CUDA(cudaStreamWaitEvent(f.prep, f.free, 0));
    if (n > 0) s = launch_preprocess(ds, cams[k], f.proj, f.prep);
    if (s == TGS_OK)
      s = launch_bin_sort(f.proj, n, W, H, gw, gh, membership, f.ws, f.ws_bytes, f.bins, f.prep,
                          F->words, F->words + 1);
    TGS_CUDA(cudaEventRecord(f.prepped, f.prep));
    // rasterize in frame order
    TGS_CUDA(cudaStreamWaitEvent(F->raster, f.prepped, 0));
    if (s == TGS_OK)
      s = c.precision == TGS_PRECISION_FP32
              ? launch_raster_fp32(f.proj, f.bins, W, H, gw, gh, o, f.rgb, f.T, nullptr, F->raster)
              : launch_raster_tc(f.proj, f.bins, W, H, gw, gh, o, f.rgb, f.T, nullptr, F->raster);
    TGS_CUDA(cudaEventRecord(f.drawn, F->raster));
    // download
    TGS_CUDA(cudaStreamWaitEvent(F->download, f.drawn, 0));
    if (s == TGS_OK) {
      TGS_CUDA(cudaMemcpyAsync(out_rgb + (size_t)k * 3 * px, f.rgb, 12 * px,
                               cudaMemcpyDeviceToHost, F->download));
      if (out_T)
        TGS_CUDA(cudaMemcpyAsync(out_T + (size_t)k * px, f.T, 4 * px, cudaMemcpyDeviceToHost,
                                 F->download));
    }
    TGS_CUDA(cudaEventRecord(f.free, F->download));
    f.used = true;
  }
  // the last rasterization of the call follows every preprocess of it (each rasterization waited
  // for its own frame's bin sort, and they run in order), so the scene copy is free after it
  TGS_CUDA(cudaEventRecord(F->scene_free[b], F->raster));
  F->scene_used[b] = true;
  TGS_CUDA(cudaEventRecord(F->done, F->download));
  // the caller's stream (NULL: the default stream) waits for the call
  TGS_CUDA(cudaStreamWaitEvent(static_cast<cudaStream_t>(stream), F->done, 0));
  ++F->calls;
  return s;
}

tgs_status tgs_frames_wait(tgs_frames* F) {
  if (!F) return set_error("null argument"), TGS_ERR_INVALID_ARGUMENT;
  Guard guard(F->device);
  TGS_CUDA(guard.status);
  TGS_CUDA(cudaEventSynchronize(F->done));
  int32_t w[2] = {0, 0};
  TGS_CUDA(cudaMemcpyAsync(w, F->words, sizeof w, cudaMemcpyDeviceToHost, F->download));
  TGS_CUDA(cudaStreamSynchronize(F->download));
  if (w[0] == 0 && w[1] == 0) return TGS_OK;
  // cleared before the call returns (every call enqueued so far has completed, so the upload
  // stream holds nothing else)
  TGS_CUDA(cudaMemsetAsync(F->words, 0, sizeof w, F->upload));
  TGS_CUDA(cudaStreamSynchronize(F->upload));
  if (w[0] != 0) {
    set_error("a bounded wait of the bin sort ran out: that frame's bins were empty");
    return TGS_ERR_TIMEOUT;
  }
  set_error("a frame needed more than %lld bin entries: its image is the background",
            (long long)F->cfg.max_entries);
  return TGS_ERR_CAPACITY;
}

tgs_status tgs_frames_destroy(tgs_frames* F) {
  if (!F) return set_error("null argument"), TGS_ERR_INVALID_ARGUMENT;
  Guard guard(F->device);
  TGS_CUDA(guard.status);
  cudaError_t e = cudaSuccess;
  for (cudaStream_t s : {F->upload, F->raster, F->download}) {
    const cudaError_t q = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = q;
  }
  for (FrameSet& f : F->sets) {
    const cudaError_t q = cudaStreamSynchronize(f.prep);
    if (e == cudaSuccess) e = q;
  }
  release(F);
  if (e != cudaSuccess) return cuda_status(e, "frames work in flight");
  return TGS_OK;
}

}  // extern "C"
