// Rendering service (tgs_serve_*): resident scenes, a worker thread and `slots` concurrent frames.
//
// The worker thread owns the slots. Each slot has its own CUDA stream, completion event and
// buffers (projected Gaussians, bins, bin-sort workspace, a T buffer when the caller passes none,
// and a pinned host word pair for the entry count and the device error word). A request is moved
// from the queue into a free slot and rendered there by the library's own calls (preprocess, bin
// sort, rasterize), all asynchronous on the slot's stream; the worker polls the slots' events, so
// frames of different requests, scenes and resolutions overlap on the GPU (continuous batching at
// request granularity). A frame whose bins overflowed the slot's capacity is rendered again after
// the capacity has grown. Scene memory and slot buffers are charged to the budget before they are
// allocated.
#include <atomic>
#include <thread>
#include <unordered_map>

#include "serve_core.h"
#include "tgs_internal.cuh"

namespace tgs {
namespace {

using serve::Clock;
using serve::Core;
using serve::Request;

constexpr int kMaxSlots = 16;
constexpr double kInitialEntriesPerGaussian = 4.0;
constexpr double kGrowth = 1.25;
constexpr int kDrainLimitMs = 10000;  // destroy: longest wait for frames still on the GPU

struct SceneRec {
  tgs_scene s{};  // device pointers into `mem`
  void* mem = nullptr;
  size_t bytes = 0;
};

struct Readback {
  int64_t num_entries;
  int32_t device_error;
  int32_t pad;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  Readback* host = nullptr;  // pinned
  // buffers and their sizes
  void* proj_mem = nullptr;
  int64_t proj_n = 0;
  tgs_projected proj{};
  void* bins_mem = nullptr;
  int64_t bins_cap = 0;
  int64_t bins_groups = 0;
  tgs_bins bins{};
  void* ws = nullptr;
  size_t ws_bytes = 0;
  float* T = nullptr;
  int64_t T_px = 0;
  size_t bytes = 0;  // device bytes charged
  // the request in flight
  bool busy = false;
  bool timed_out = false;
  Request req{};
  int64_t scene_n = 0;
};

inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

size_t projected_bytes(int64_t n) {
  return a256(8 * n) + a256(16 * n) + a256(12 * n) + a256(4 * n) + a256(4 * n) + a256(16 * n);
}

size_t bins_bytes(int64_t cap, int64_t groups) {
  return a256(4 * cap) + a256(2 * cap) + a256(8 * groups) + a256(8);
}

}  // namespace
}  // namespace tgs

struct tgs_server {
  tgs_serve_config cfg{};
  tgs::serve::Core core;
  std::thread worker;
  std::mutex scene_mu;
  std::unordered_map<int32_t, tgs::SceneRec> scenes;
  int32_t next_scene = 0;
  std::atomic<int64_t> hbm{0};
  std::atomic<int64_t> regrown{0};
  std::vector<tgs::Slot> slots;
  std::atomic<bool> drained{true};
  int32_t* err_word = nullptr;

  explicit tgs_server(const tgs_serve_config& c) : cfg(c), core(c.max_inflight, c.request_timeout_ms) {}

  // Charges `bytes` to the budget; false if they do not fit.
  bool reserve(size_t bytes) {
    int64_t cur = hbm.load();
    while (true) {
      if (cur + (int64_t)bytes > cfg.hbm_budget_bytes) return false;
      if (hbm.compare_exchange_weak(cur, cur + (int64_t)bytes)) return true;
    }
  }
  void unreserve(size_t bytes) { hbm.fetch_sub((int64_t)bytes); }
};

namespace tgs {
namespace {

void free_slot_buffers(tgs_server* S, Slot& sl) {
  cudaFree(sl.proj_mem);
  cudaFree(sl.bins_mem);
  cudaFree(sl.ws);
  cudaFree(sl.T);
  sl.proj_mem = sl.bins_mem = sl.ws = nullptr;
  sl.T = nullptr;
  sl.proj_n = sl.bins_cap = sl.bins_groups = sl.T_px = 0;
  sl.ws_bytes = 0;
  S->unreserve(sl.bytes);
  sl.bytes = 0;
}

// Makes the slot's buffers large enough for n Gaussians, `cap` bin entries, the image and (if the
// caller gave no T buffer) a T image. Buffers only grow; a grown buffer is reallocated (the slot
// is idle). Returns TGS_ERR_CAPACITY if the budget cannot hold them.
tgs_status ensure_buffers(tgs_server* S, Slot& sl, int64_t n, int64_t cap, const tgs_camera& cam,
                          bool need_T) {
  const int TX = div_up(cam.width, kTile), TY = div_up(cam.height, kTile);
  const int64_t groups =
      (int64_t)div_up(TX, S->cfg.tiling.group_w) * div_up(TY, S->cfg.tiling.group_h);
  size_t ws_need = 0;
  tgs_status s = tgs_bin_sort_workspace_size(n, cap, cam.width, cam.height, &S->cfg.tiling, &ws_need);
  if (s != TGS_OK) return s;
  const int64_t px = need_T ? (int64_t)cam.width * cam.height : 0;
  // Replaces *mem (old_bytes) by a buffer of new_bytes. The new size is charged first; if it does
  // not fit, nothing changes. *lost tells whether the old buffer is gone (a failed allocation).
  bool lost = false;
  auto grow = [&](void** mem, size_t old_bytes, size_t new_bytes) -> tgs_status {
    lost = false;
    if (!S->reserve(new_bytes)) {
      set_error("serving budget of %lld bytes exceeded", (long long)S->cfg.hbm_budget_bytes);
      return TGS_ERR_CAPACITY;
    }
    cudaFree(*mem);
    *mem = nullptr;
    lost = true;
    S->unreserve(old_bytes);
    sl.bytes -= old_bytes;
    const cudaError_t e = device_malloc(mem, new_bytes);
    if (e != cudaSuccess) {
      S->unreserve(new_bytes);
      return cuda_status(e, "cudaMalloc (serving slot)");
    }
    sl.bytes += new_bytes;
    return TGS_OK;
  };
  if (n > sl.proj_n) {
    s = grow(&sl.proj_mem, sl.proj_n ? projected_bytes(sl.proj_n) : 0, projected_bytes(n));
    if (s != TGS_OK) {
      if (lost) sl.proj_n = 0;
      return s;
    }
    sl.proj_n = n;
    char* p = static_cast<char*>(sl.proj_mem);
    size_t off = 0;
    auto take = [&](size_t b) { char* q = p + off; off += a256(b); return q; };
    sl.proj.mean2d = reinterpret_cast<float*>(take(8 * n));
    sl.proj.conic_opacity = reinterpret_cast<float*>(take(16 * n));
    sl.proj.rgb = reinterpret_cast<float*>(take(12 * n));
    sl.proj.depth = reinterpret_cast<float*>(take(4 * n));
    sl.proj.radius = reinterpret_cast<int32_t*>(take(4 * n));
    sl.proj.rect = reinterpret_cast<int32_t*>(take(16 * n));
  }
  if (cap > sl.bins_cap || groups > sl.bins_groups) {
    const int64_t nc = std::max(cap, sl.bins_cap), ng = std::max(groups, sl.bins_groups);
    s = grow(&sl.bins_mem, sl.bins_cap ? bins_bytes(sl.bins_cap, sl.bins_groups) : 0,
             bins_bytes(nc, ng));
    if (s != TGS_OK) {
      if (lost) sl.bins_cap = sl.bins_groups = 0;
      return s;
    }
    sl.bins_cap = nc;
    sl.bins_groups = ng;
    char* p = static_cast<char*>(sl.bins_mem);
    size_t off = 0;
    auto take = [&](size_t b) { char* q = p + off; off += a256(b); return q; };
    sl.bins.capacity = nc;
    sl.bins.keys = nullptr;
    sl.bins.vals = reinterpret_cast<uint32_t*>(take(4 * nc));
    sl.bins.masks = reinterpret_cast<uint16_t*>(take(2 * nc));
    sl.bins.ranges = reinterpret_cast<uint32_t*>(take(8 * ng));
    sl.bins.num_entries = reinterpret_cast<int64_t*>(take(8));
  }
  if (ws_need > sl.ws_bytes) {
    s = grow(&sl.ws, sl.ws_bytes, ws_need);
    if (s != TGS_OK) {
      if (lost) sl.ws_bytes = 0;
      return s;
    }
    sl.ws_bytes = ws_need;
  }
  if (px > sl.T_px) {
    void* m = sl.T;
    s = grow(&m, 4 * (size_t)sl.T_px, 4 * (size_t)px);
    sl.T = static_cast<float*>(m);
    if (s != TGS_OK) {
      if (lost) sl.T_px = 0;
      return s;
    }
    sl.T_px = px;
  }
  return TGS_OK;
}

// Enqueues the frame of the slot's request on its stream. On failure the caller completes it.
tgs_status issue(tgs_server* S, Slot& sl) {
  const Request& r = sl.req;
  tgs_scene scene;
  {
    std::lock_guard<std::mutex> lock(S->scene_mu);
    auto it = S->scenes.find(r.scene);
    if (it == S->scenes.end()) return set_error("scene %d was removed", r.scene), TGS_ERR_NOT_FOUND;
    scene = it->second.s;  // kept alive by the request's scene reference
  }
  sl.scene_n = scene.n;
  const int64_t want = std::max<int64_t>(
      sl.bins_cap, (int64_t)(kInitialEntriesPerGaussian * (double)scene.n) + 4096);
  tgs_status s = ensure_buffers(S, sl, std::max<int64_t>(scene.n, 1), want, r.camera, !r.out_T);
  if (s != TGS_OK) return s;
  cudaStream_t st = sl.stream;
  s = tgs_preprocess(&scene, &r.camera, &sl.proj, st);
  if (s != TGS_OK) return s;
  s = tgs_bin_sort(&sl.proj, scene.n, r.camera.width, r.camera.height, &S->cfg.tiling, sl.ws,
                   sl.ws_bytes, &sl.bins, nullptr, st);
  if (s != TGS_OK) return s;
  tgs_raster_opts o{};
  o.precision = S->cfg.precision;
  o.flags = 0;
  o.bg[0] = S->cfg.bg[0];
  o.bg[1] = S->cfg.bg[1];
  o.bg[2] = S->cfg.bg[2];
  o.counters = nullptr;
  s = tgs_rasterize(&sl.proj, scene.n, &sl.bins, r.camera.width, r.camera.height, &S->cfg.tiling, &o,
                    r.out_rgb, r.out_T ? r.out_T : sl.T, nullptr, st);
  if (s != TGS_OK) return s;
  TGS_CUDA(cudaMemcpyAsync(&sl.host->num_entries, sl.bins.num_entries, sizeof(int64_t),
                           cudaMemcpyDeviceToHost, st));
  TGS_CUDA(cudaMemcpyAsync(&sl.host->device_error, S->err_word, sizeof(int32_t),
                           cudaMemcpyDeviceToHost, st));
  TGS_CUDA(cudaEventRecord(sl.done, st));
  return TGS_OK;
}

// The request leaves its slot: released first, so that a client woken by the completion already
// sees its scene free and its admission returned.
void finish(tgs_server* S, Slot& sl, tgs_status st) {
  S->core.release(sl.req);
  S->core.complete(sl.req.ticket, st);
  sl.busy = false;
  sl.timed_out = false;
}

// Handles a slot whose event has completed.
void on_done(tgs_server* S, Slot& sl) {
  if (sl.host->device_error != TGS_OK) {
    // a bounded device wait expired in this frame (the error word is shared by the device)
    cudaMemsetAsync(S->err_word, 0, sizeof(int32_t), sl.stream);
    finish(S, sl, TGS_ERR_TIMEOUT);
    return;
  }
  const int64_t need = sl.host->num_entries;
  if (need > sl.bins_cap && !sl.timed_out) {  // overflow: grow and render again
    const int64_t cap = (int64_t)(kGrowth * (double)need) + 4096;
    tgs_status s = ensure_buffers(S, sl, std::max<int64_t>(sl.scene_n, 1), cap, sl.req.camera,
                                  !sl.req.out_T);
    if (s == TGS_OK) s = issue(S, sl);
    if (s != TGS_OK) {
      finish(S, sl, s);
      return;
    }
    S->regrown.fetch_add(1);
    return;  // still busy
  }
  finish(S, sl, need > sl.bins_cap ? TGS_ERR_CAPACITY : TGS_OK);
}

void worker_main(tgs_server* S) {
  cudaSetDevice(S->cfg.device);
  Clock::time_point stop_seen{};
  while (true) {
    bool progress = false, any_busy = false;
    const auto now = Clock::now();
    for (Slot& sl : S->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaSuccess) {
        on_done(S, sl);
        progress = true;
      } else if (q != cudaErrorNotReady) {
        cuda_status(q, "serving frame");
        finish(S, sl, TGS_ERR_CUDA);
        progress = true;
      } else if (!sl.timed_out && S->core.expired(sl.req, now)) {
        S->core.complete(sl.req.ticket, TGS_ERR_TIMEOUT);  // the slot stays busy until the GPU is done
        sl.timed_out = true;
      }
      any_busy |= sl.busy;
    }
    const bool stopping = S->core.stopping();
    if (!stopping) {
      for (Slot& sl : S->slots) {
        if (sl.busy) continue;
        Request r;
        if (!S->core.next(&r)) break;
        sl.req = r;
        sl.busy = true;
        sl.timed_out = false;
        const tgs_status s = issue(S, sl);
        if (s != TGS_OK) finish(S, sl, s);
        any_busy |= sl.busy;
        progress = true;
      }
    } else {
      if (!any_busy) break;
      if (stop_seen == Clock::time_point{}) stop_seen = now;
      if (now - stop_seen > std::chrono::milliseconds(kDrainLimitMs)) {
        S->drained.store(false);  // frames still on the GPU: their buffers are not freed
        break;
      }
    }
    if (!progress) {
      if (any_busy)
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      else if (!stopping)
        S->core.wait_for_work(20);
    }
  }
}

// Makes `dev` current for the scope and restores the caller's device afterwards.
struct DeviceGuard {
  int prev = -1;
  cudaError_t status;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    status = cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

bool valid_camera(const tgs_camera* c) {
  return c && c->width >= 1 && c->height >= 1 && c->width <= 16384 && c->height <= 16384 &&
         c->fx > 0 && c->fy > 0;
}

}  // namespace
}  // namespace tgs

using namespace tgs;

extern "C" {

tgs_status tgs_serve_create(const tgs_serve_config* config, tgs_server** out) {
  if (!config || !out) return set_error("null argument"), TGS_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  const tgs_serve_config& c = *config;
  if (c.max_inflight < 1 || c.slots < 1 || c.slots > kMaxSlots || c.hbm_budget_bytes <= 0 ||
      (c.precision != TGS_PRECISION_FP32 && c.precision != TGS_PRECISION_FP16_TC &&
       c.precision != TGS_PRECISION_BF16_TC) ||
      c.tiling.group_w < 1 || c.tiling.group_w > TGS_MAX_GROUP || c.tiling.group_h < 1 ||
      c.tiling.group_h > TGS_MAX_GROUP || (c.tiling.flags & ~TGS_BIN_RANGE_ONLY) != 0 ||
      c.request_timeout_ms < 0)
    return set_error("bad serving config"), TGS_ERR_INVALID_ARGUMENT;
  tgs_status s = tgs_check_device(c.device);
  if (s != TGS_OK) return s;
  DeviceGuard guard(c.device);
  TGS_CUDA(guard.status);
  int32_t* err = device_error_word();
  if (!err) return set_error("device error word unavailable"), TGS_ERR_CUDA;
  auto* S = new tgs_server(c);
  S->err_word = err;
  S->slots.resize(c.slots);
  for (Slot& sl : S->slots) {
    cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = pinned_malloc(reinterpret_cast<void**>(&sl.host), sizeof(Readback));
    if (e != cudaSuccess) {
      for (Slot& t : S->slots) {
        if (t.stream) cudaStreamDestroy(t.stream);
        if (t.done) cudaEventDestroy(t.done);
        if (t.host) cudaFreeHost(t.host);
      }
      delete S;
      return cuda_status(e, "serving slot");
    }
  }
  S->worker = std::thread(worker_main, S);
  *out = S;
  return TGS_OK;
}

tgs_status tgs_serve_add_scene(tgs_server* S, const tgs_scene* scene, int32_t* scene_id) {
  if (!S || !scene || !scene_id) return set_error("null argument"), TGS_ERR_INVALID_ARGUMENT;
  const int64_t n = scene->n;
  if (n < 0 || n >= (int64_t(1) << 30) || scene->sh_degree < 0 || scene->sh_degree > 3)
    return set_error("bad scene"), TGS_ERR_INVALID_ARGUMENT;
  if (n > 0 && (!scene->means || !scene->scales || !scene->quats || !scene->opacities || !scene->sh))
    return set_error("null scene array"), TGS_ERR_INVALID_ARGUMENT;
  const int64_t k = (int64_t)(scene->sh_degree + 1) * (scene->sh_degree + 1);
  const size_t b_means = a256(12 * n), b_scales = a256(12 * n), b_quats = a256(16 * n),
               b_opac = a256(4 * n), b_sh = a256(12 * k * n);
  const size_t bytes = std::max<size_t>(256, b_means + b_scales + b_quats + b_opac + b_sh);
  if (!S->reserve(bytes)) {
    set_error("serving budget of %lld bytes exceeded by a scene of %zu bytes",
              (long long)S->cfg.hbm_budget_bytes, bytes);
    return TGS_ERR_CAPACITY;
  }
  DeviceGuard guard(S->cfg.device);
  TGS_CUDA(guard.status);
  SceneRec rec;
  cudaError_t e = device_malloc(&rec.mem, bytes);
  if (e != cudaSuccess) {
    S->unreserve(bytes);
    return cuda_status(e, "cudaMalloc (scene)");
  }
  rec.bytes = bytes;
  char* p = static_cast<char*>(rec.mem);
  float* d_means = reinterpret_cast<float*>(p);
  float* d_scales = reinterpret_cast<float*>(p + b_means);
  float* d_quats = reinterpret_cast<float*>(p + b_means + b_scales);
  float* d_opac = reinterpret_cast<float*>(p + b_means + b_scales + b_quats);
  float* d_sh = reinterpret_cast<float*>(p + b_means + b_scales + b_quats + b_opac);
  rec.s = *scene;
  rec.s.means = d_means;
  rec.s.scales = d_scales;
  rec.s.quats = d_quats;
  rec.s.opacities = d_opac;
  rec.s.sh = d_sh;
  if (n > 0) {
    const struct { const float* src; float* dst; size_t bytes; } copies[] = {
        {scene->means, d_means, 12 * (size_t)n},
        {scene->scales, d_scales, 12 * (size_t)n},
        {scene->quats, d_quats, 16 * (size_t)n},
        {scene->opacities, d_opac, 4 * (size_t)n},
        {scene->sh, d_sh, 12 * (size_t)k * (size_t)n}};
    for (const auto& c : copies) {
      e = cudaMemcpy(c.dst, c.src, c.bytes, cudaMemcpyDefault);
      if (e != cudaSuccess) {
        cudaFree(rec.mem);
        S->unreserve(bytes);
        return cuda_status(e, "cudaMemcpy (scene)");
      }
    }
  }
  std::lock_guard<std::mutex> lock(S->scene_mu);
  const int32_t id = S->next_scene++;
  S->scenes[id] = rec;
  *scene_id = id;
  return TGS_OK;
}

tgs_status tgs_serve_remove_scene(tgs_server* S, int32_t scene_id) {
  if (!S) return set_error("null server"), TGS_ERR_INVALID_ARGUMENT;
  SceneRec rec;
  {
    std::lock_guard<std::mutex> lock(S->scene_mu);
    auto it = S->scenes.find(scene_id);
    if (it == S->scenes.end()) return set_error("unknown scene %d", scene_id), TGS_ERR_NOT_FOUND;
    if (S->core.scene_refs(scene_id) > 0)
      return set_error("scene %d has requests in flight", scene_id), TGS_ERR_BUSY;
    rec = it->second;
    S->scenes.erase(it);
  }
  DeviceGuard guard(S->cfg.device);
  cudaFree(rec.mem);
  S->unreserve(rec.bytes);
  return TGS_OK;
}

tgs_status tgs_serve_submit(tgs_server* S, int32_t scene_id, const tgs_camera* camera,
                            float* out_rgb, float* out_T, uint64_t* ticket) {
  if (!S || !ticket || !out_rgb || !valid_camera(camera))
    return set_error("bad argument"), TGS_ERR_INVALID_ARGUMENT;
  Request r;
  r.scene = scene_id;
  r.camera = *camera;
  r.out_rgb = out_rgb;
  r.out_T = out_T;
  // the scene lock keeps remove_scene from freeing it between the check and the admission
  std::lock_guard<std::mutex> lock(S->scene_mu);
  if (S->scenes.find(scene_id) == S->scenes.end())
    return set_error("unknown scene %d", scene_id), TGS_ERR_NOT_FOUND;
  const tgs_status s = S->core.submit(r, ticket);
  if (s == TGS_ERR_BUSY) set_error("serving queue full (max_inflight %d)", S->cfg.max_inflight);
  return s;
}

tgs_status tgs_serve_poll(tgs_server* S, uint64_t ticket, int32_t* done, tgs_status* result) {
  if (!S || !done) return set_error("null argument"), TGS_ERR_INVALID_ARGUMENT;
  return S->core.poll(ticket, done, result);
}

tgs_status tgs_serve_wait(tgs_server* S, uint64_t ticket, int32_t timeout_ms, tgs_status* result) {
  if (!S) return set_error("null server"), TGS_ERR_INVALID_ARGUMENT;
  return S->core.wait(ticket, timeout_ms, result);
}

tgs_status tgs_serve_pause(tgs_server* S, int32_t paused) {
  if (!S) return set_error("null server"), TGS_ERR_INVALID_ARGUMENT;
  S->core.set_paused(paused != 0);
  return TGS_OK;
}

tgs_status tgs_serve_get_stats(tgs_server* S, tgs_serve_stats* out) {
  if (!S || !out) return set_error("null argument"), TGS_ERR_INVALID_ARGUMENT;
  S->core.stats(out);
  out->regrown = S->regrown.load();
  out->hbm_bytes = S->hbm.load();
  return TGS_OK;
}

tgs_status tgs_serve_destroy(tgs_server* S) {
  if (!S) return set_error("null server"), TGS_ERR_INVALID_ARGUMENT;
  S->core.stop();
  if (S->worker.joinable()) S->worker.join();
  DeviceGuard guard(S->cfg.device);
  const bool drained = S->drained.load();
  for (Slot& sl : S->slots) {
    if (drained) {  // else frames may still write to these buffers: they are left allocated
      free_slot_buffers(S, sl);
      cudaFreeHost(sl.host);
    }
    cudaStreamDestroy(sl.stream);
    cudaEventDestroy(sl.done);
  }
  if (drained)
    for (auto& kv : S->scenes) cudaFree(kv.second.mem);
  delete S;
  if (!drained)
    return set_error("frames still running after %d ms: their device memory was not freed",
                     kDrainLimitMs),
           TGS_ERR_TIMEOUT;
  return TGS_OK;
}

}  // extern "C"
