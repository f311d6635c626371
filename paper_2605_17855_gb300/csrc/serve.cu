// Rendering service (tgs_serve_*): resident scenes, a worker thread, `slots` concurrent frames
// and batched tensor-core rasterization.
//
// Every device buffer is allocated on the client's thread: one block per slot at creation (sized
// for max_gaussians, max_width x max_height and max_entries) and one block per scene; the worker
// thread allocates nothing. Each slot has its own stream, its buffers (projected Gaussians, bins,
// bin-sort workspace, a T image for requests that bring none) and three device words: a readiness
// flag, a status word and the bin sort's error word.
//
// The worker moves queued requests into free slots and preprocesses and bins them there,
// asynchronously on the slot's stream (frames of different scenes and resolutions overlap on the
// GPU). With a tensor-core precision, the slots whose binning has finished are then rasterized
// together by one persistent launch (tgs_rasterize_batch over (frame, tile group) work items). Up
// to two launches are in flight, each on its own stream with half of the GPU's CTA slots, so a
// launch of newly binned frames starts beside a running one; requests that arrive meanwhile are
// binned and join the next launch (continuous batching). The launch waits (bounded) on each slot's
// readiness flag, which the slot's stream raises after binning, and reports a time-out to that
// slot's status word only. With FP32 each slot rasterizes on its own stream.
#include <algorithm>
#include <atomic>
#include <thread>
#include <unordered_map>

#include "groupings.h"
#include "serve_core.h"
#include "tgs_internal.cuh"

namespace tgs {
namespace {

using serve::Clock;
using serve::Core;
using serve::Request;

constexpr int kMaxSlots = 16;
constexpr int kMaxBatches = 2;              // batched launches in flight
constexpr int kDrainLimitMs = 10000;        // destroy: longest wait for frames still on the GPU
constexpr uint64_t kReadyWaitNs = 2000000000ull;

struct SceneRec {
  tgs_scene s{};  // device pointers into `mem`
  void* mem = nullptr;
  size_t bytes = 0;
};

// Pinned host words of a slot. num_entries and sort_error are copied back after binning; status
// and done are written by the batched launch itself (pinned memory is mapped into the device's
// address space), so the worker sees a frame finish as soon as its last tile group is rendered.
struct Readback {
  int64_t num_entries;
  int32_t sort_error;  // the bin sort's error word
  int32_t status;      // the frame's status word in the batched launch
  int32_t done;        // set to the slot's sequence number when the frame is complete
  int32_t pad;
};

enum class SlotState { kFree, kBinning, kReady, kRaster };

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;  // binning done (tensor cores) or frame done (FP32)
  Readback* host = nullptr;    // pinned
  void* mem = nullptr;         // every device buffer of the slot
  tgs_projected proj{};
  tgs_bins bins{};
  void* ws = nullptr;
  size_t ws_bytes = 0;
  float* T = nullptr;
  int32_t* words = nullptr;    // [0] readiness flag, [1] status, [2] bin-sort error word
  int32_t seq = 0;             // value of the readiness flag for the request in the slot
  SlotState state = SlotState::kFree;
  int batch = -1;  // the batched launch rasterizing the slot's frame
  bool timed_out = false;
  Request req{};
  int64_t scene_n = 0;
};

struct Batch {
  cudaStream_t stream = nullptr;  // each launch its own stream: two run side by side
  cudaEvent_t done = nullptr;
  int* counter = nullptr;  // device work counter (tgs_rasterize_batch workspace)
  std::vector<int> slots;
  bool busy = false;
};

inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

__global__ void k_set_flag(int32_t* flag, int32_t value) { *flag = value; }

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
  std::vector<tgs::Slot> slots;
  tgs::Batch batches[tgs::kMaxBatches];
  void* batch_mem = nullptr;
  size_t slot_bytes = 0;
  std::atomic<bool> drained{true};

  explicit tgs_server(const tgs_serve_config& c) : cfg(c), core(c.max_inflight, c.request_timeout_ms) {}

  bool tensor_cores() const { return cfg.precision != TGS_PRECISION_FP32; }

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

int64_t max_groups(const tgs_serve_config& c) {
  return (int64_t)div_up(div_up(c.max_width, kTile), c.tiling.group_w) *
         div_up(div_up(c.max_height, kTile), c.tiling.group_h);
}

// Bytes of one slot's buffers, and their layout inside the slot's block when `sl` is given.
size_t slot_layout(const tgs_serve_config& c, Slot* sl) {
  const int64_t n = c.max_gaussians, cap = c.max_entries, G = max_groups(c);
  const int GX = div_up(div_up(c.max_width, kTile), c.tiling.group_w);
  const int GY = div_up(div_up(c.max_height, kTile), c.tiling.group_h);
  const size_t ws = bin_sort_workspace_bytes(n, cap, GX, GY);
  char* p = sl ? static_cast<char*>(sl->mem) : nullptr;
  size_t off = 0;
  auto take = [&](size_t b) {
    char* q = p ? p + off : nullptr;
    off += a256(b);
    return q;
  };
  char* mean2d = take(8 * n);
  char* conic = take(16 * n);
  char* rgb = take(12 * n);
  char* depth = take(4 * n);
  char* radius = take(4 * n);
  char* rect = take(16 * n);
  char* vals = take(4 * cap);
  char* masks = take(2 * cap);
  char* ranges = take(8 * G);
  char* count = take(8);
  char* wsp = take(ws);
  char* T = take(4 * (size_t)c.max_width * c.max_height);
  char* words = take(16);
  if (sl) {
    sl->proj.mean2d = reinterpret_cast<float*>(mean2d);
    sl->proj.conic_opacity = reinterpret_cast<float*>(conic);
    sl->proj.rgb = reinterpret_cast<float*>(rgb);
    sl->proj.depth = reinterpret_cast<float*>(depth);
    sl->proj.radius = reinterpret_cast<int32_t*>(radius);
    sl->proj.rect = reinterpret_cast<int32_t*>(rect);
    sl->bins.capacity = cap;
    sl->bins.keys = nullptr;
    sl->bins.vals = reinterpret_cast<uint32_t*>(vals);
    sl->bins.masks = reinterpret_cast<uint16_t*>(masks);
    sl->bins.ranges = reinterpret_cast<uint32_t*>(ranges);
    sl->bins.num_entries = reinterpret_cast<int64_t*>(count);
    sl->ws = wsp;
    sl->ws_bytes = ws;
    sl->T = reinterpret_cast<float*>(T);
    sl->words = reinterpret_cast<int32_t*>(words);
  }
  return off;
}

// Enqueues preprocess + bin sort of the slot's request on its stream (and, with FP32, the
// rasterization). On failure the caller completes the request.
tgs_status issue(tgs_server* S, Slot& sl) {
  const Request& r = sl.req;
  tgs_scene scene;
  {
    std::lock_guard<std::mutex> lock(S->scene_mu);
    auto it = S->scenes.find(r.scene);
    if (it == S->scenes.end()) return set_error("scene %d was removed", r.scene), TGS_ERR_NOT_FOUND;
    scene = it->second.s;  // kept alive by the request's scene reference
  }
  if (r.camera.width > S->cfg.max_width || r.camera.height > S->cfg.max_height)
    return set_error("a %dx%d frame exceeds the slots' %dx%d", r.camera.width, r.camera.height,
                     S->cfg.max_width, S->cfg.max_height),
           TGS_ERR_CAPACITY;
  sl.scene_n = scene.n;
  cudaStream_t st = sl.stream;
  ++sl.seq;
  TGS_CUDA(cudaMemsetAsync(sl.words + 1, 0, 2 * sizeof(int32_t), st));  // status, error word
  tgs_status s = TGS_OK;
  if (scene.n > 0) {
    s = launch_preprocess(scene, r.camera, sl.proj, st);
    if (s != TGS_OK) return s;
  }
  s = launch_bin_sort(sl.proj, scene.n, r.camera.width, r.camera.height, S->cfg.tiling.group_w,
                      S->cfg.tiling.group_h, (S->cfg.tiling.flags & TGS_BIN_RANGE_ONLY) == 0, sl.ws,
                      sl.ws_bytes, sl.bins, st, sl.words + 2);
  if (s != TGS_OK) return s;
  if (!S->tensor_cores()) {
    tgs_raster_opts o{};
    o.precision = TGS_PRECISION_FP32;
    for (int k = 0; k < 3; ++k) o.bg[k] = S->cfg.bg[k];
    s = launch_raster_fp32(sl.proj, sl.bins, r.camera.width, r.camera.height, S->cfg.tiling.group_w,
                           S->cfg.tiling.group_h, o, r.out_rgb, r.out_T ? r.out_T : sl.T, nullptr, st);
    if (s != TGS_OK) return s;
  } else {
    k_set_flag<<<1, 1, 0, st>>>(sl.words, sl.seq);
    TGS_CHECK_LAUNCH("k_set_flag");
  }
  TGS_CUDA(cudaMemcpyAsync(&sl.host->num_entries, sl.bins.num_entries, sizeof(int64_t),
                           cudaMemcpyDeviceToHost, st));
  TGS_CUDA(cudaMemcpyAsync(&sl.host->sort_error, sl.words + 2, sizeof(int32_t), cudaMemcpyDeviceToHost,
                           st));
  TGS_CUDA(cudaEventRecord(sl.done, st));
  sl.state = SlotState::kBinning;
  return TGS_OK;
}

// The request leaves its slot: released first, so that a client woken by the completion already
// sees its scene free and its admission returned.
void finish(tgs_server* S, Slot& sl, tgs_status st) {
  S->core.release(sl.req);
  S->core.complete(sl.req.ticket, st);
  sl.state = SlotState::kFree;
  sl.batch = -1;
  sl.timed_out = false;
}

int32_t host_word(const int32_t* w) { return *reinterpret_cast<const volatile int32_t*>(w); }

// Status of a frame whose binning (and, with FP32, rasterization) has completed.
tgs_status binning_status(const tgs_server* S, const Slot& sl) {
  if (sl.host->sort_error != TGS_OK) return TGS_ERR_TIMEOUT;
  if (sl.host->num_entries > S->cfg.max_entries) return TGS_ERR_CAPACITY;
  return TGS_OK;
}

// Rasterizes every binned slot with one persistent tensor-core launch on the batch stream, the
// frames ordered from the fewest pixels to the most (small frames complete first).
tgs_status launch_batch(tgs_server* S, int bi) {
  Batch& b = S->batches[bi];
  b.slots.clear();
  for (int k = 0; k < (int)S->slots.size(); ++k)
    if (S->slots[k].state == SlotState::kReady) b.slots.push_back(k);
  if (b.slots.empty()) return TGS_OK;
  auto pixels = [&](int k) {
    const tgs_camera& c = S->slots[k].req.camera;
    return (int64_t)c.width * c.height;
  };
  std::stable_sort(b.slots.begin(), b.slots.end(), [&](int x, int y) { return pixels(x) < pixels(y); });
  RasterFrame rf[kMaxSlots];
  int count = 0;
  for (int k : b.slots) {
    Slot& sl = S->slots[k];
    TGS_CUDA(cudaStreamWaitEvent(b.stream, sl.done, 0));
    sl.host->status = TGS_OK;
    sl.host->done = 0;
    const Request& r = sl.req;
    rf[count++] = RasterFrame{&sl.proj, &sl.bins, r.camera.width, r.camera.height, r.out_rgb,
                              r.out_T ? r.out_T : sl.T, sl.words, sl.seq, &sl.host->status,
                              &sl.host->done, sl.seq};
  }
  tgs_raster_opts o{};
  o.precision = S->cfg.precision;
  for (int k = 0; k < 3; ++k) o.bg[k] = S->cfg.bg[k];
  // each launch takes at most half of the GPU's CTA slots, so that a launch of newly binned
  // (often small) frames starts beside a running one instead of queueing behind it
  tgs_status s = launch_raster_tc_batch(rf, count, S->cfg.tiling.group_w, S->cfg.tiling.group_h, o,
                                        b.counter, kReadyWaitNs, b.stream, kMaxBatches);
  if (s != TGS_OK) {
    b.slots.clear();
    return s;
  }
  for (int k : b.slots) {
    S->slots[k].state = SlotState::kRaster;
    S->slots[k].batch = bi;
  }
  TGS_CUDA(cudaEventRecord(b.done, b.stream));
  b.busy = true;
  return TGS_OK;
}

void worker_main(tgs_server* S) {
  cudaSetDevice(S->cfg.device);
  Clock::time_point stop_seen{};
  while (true) {
    bool progress = false, any_busy = false;
    const auto now = Clock::now();
    // frames whose last tile group the batched launch has rendered
    for (Slot& sl : S->slots) {
      if (sl.state != SlotState::kRaster || host_word(&sl.host->done) != sl.seq) continue;
      finish(S, sl, host_word(&sl.host->status) == TGS_OK ? TGS_OK : TGS_ERR_TIMEOUT);
      progress = true;
    }
    // batched launches that ended: any frame of theirs not reported done failed (a CTA gave up)
    for (int bi = 0; bi < kMaxBatches; ++bi) {
      Batch& b = S->batches[bi];
      if (!b.busy) continue;
      const cudaError_t q = cudaEventQuery(b.done);
      if (q == cudaErrorNotReady) continue;
      for (int k : b.slots) {
        Slot& sl = S->slots[k];
        if (sl.state != SlotState::kRaster || sl.batch != bi) continue;
        if (q != cudaSuccess) {
          cuda_status(q, "batched rasterization");
          finish(S, sl, TGS_ERR_CUDA);
        } else {
          const bool ok = host_word(&sl.host->done) == sl.seq && host_word(&sl.host->status) == TGS_OK;
          finish(S, sl, ok ? TGS_OK : TGS_ERR_TIMEOUT);
        }
      }
      b.busy = false;
      b.slots.clear();
      progress = true;
    }
    // slots whose binning (or FP32 frame) completed
    for (Slot& sl : S->slots) {
      if (sl.state == SlotState::kFree) continue;
      any_busy = true;
      if (sl.state == SlotState::kBinning) {
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaSuccess) {
          const tgs_status st = binning_status(S, sl);
          if (st != TGS_OK || !S->tensor_cores() || sl.timed_out)
            finish(S, sl, st);
          else
            sl.state = SlotState::kReady;
          progress = true;
        } else if (q != cudaErrorNotReady) {
          cuda_status(q, "serving frame");
          finish(S, sl, TGS_ERR_CUDA);
          progress = true;
        }
      }
      if (sl.state != SlotState::kFree && !sl.timed_out && S->core.expired(sl.req, now)) {
        S->core.complete(sl.req.ticket, TGS_ERR_TIMEOUT);  // the slot stays busy until the GPU is done
        sl.timed_out = true;
      }
    }
    const bool stopping = S->core.stopping();
    if (!stopping) {
      for (Slot& sl : S->slots) {
        if (sl.state != SlotState::kFree) continue;
        Request r;
        if (!S->core.next(&r)) break;
        sl.req = r;
        sl.timed_out = false;
        const tgs_status s = issue(S, sl);
        if (s != TGS_OK) finish(S, sl, s);
        any_busy |= sl.state != SlotState::kFree;
        progress = true;
      }
    }
    // one persistent launch over every binned frame, if a launch slot is free
    bool ready = false;
    for (Slot& sl : S->slots) ready |= sl.state == SlotState::kReady;
    if (ready) {
      for (int bi = 0; bi < kMaxBatches; ++bi) {
        if (S->batches[bi].busy) continue;
        const tgs_status s = launch_batch(S, bi);
        if (s != TGS_OK)
          for (Slot& sl : S->slots)
            if (sl.state == SlotState::kReady) finish(S, sl, s);
        progress = true;
        break;
      }
    }
    if (stopping) {
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
      !grouping_supported(c.precision, c.tiling.group_w, c.tiling.group_h) ||
      (c.tiling.flags & ~TGS_BIN_RANGE_ONLY) != 0 ||
      c.request_timeout_ms < 0 || c.max_gaussians < 1 || c.max_gaussians >= (int64_t(1) << 30) ||
      c.max_width < 1 || c.max_width > 16384 || c.max_height < 1 || c.max_height > 16384 ||
      c.max_entries < 1 || c.max_entries >= (int64_t(1) << 30))
    return set_error("bad serving config"), TGS_ERR_INVALID_ARGUMENT;
  tgs_status s = tgs_check_device(c.device);
  if (s != TGS_OK) return s;
  DeviceGuard guard(c.device);
  TGS_CUDA(guard.status);
  auto* S = new tgs_server(c);
  S->slot_bytes = slot_layout(c, nullptr);
  const size_t batch_bytes = 256 * kMaxBatches;
  const size_t total = S->slot_bytes * (size_t)c.slots + batch_bytes;
  if (!S->reserve(total)) {
    set_error("%d slots of %zu bytes exceed the serving budget of %lld bytes", c.slots, S->slot_bytes,
              (long long)c.hbm_budget_bytes);
    delete S;
    return TGS_ERR_CAPACITY;
  }
  // stream priorities: the slots' short binning kernels take SM slots as the batched launch's CTAs
  // retire, instead of queueing behind it
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  auto cleanup = [&](cudaError_t e, const char* what) {
    for (Slot& t : S->slots) {
      if (t.stream) cudaStreamDestroy(t.stream);
      if (t.done) cudaEventDestroy(t.done);
      if (t.host) cudaFreeHost(t.host);
      if (t.mem) cudaFree(t.mem);
    }
    for (Batch& b : S->batches) {
      if (b.done) cudaEventDestroy(b.done);
      if (b.stream) cudaStreamDestroy(b.stream);
    }
    if (S->batch_mem) cudaFree(S->batch_mem);
    delete S;
    return cuda_status(e, what);
  };
  S->slots.resize(c.slots);
  for (Slot& sl : S->slots) {
    cudaError_t e = cudaStreamCreateWithPriority(&sl.stream, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = pinned_malloc(reinterpret_cast<void**>(&sl.host), sizeof(Readback));
    if (e == cudaSuccess) e = device_malloc(&sl.mem, S->slot_bytes);
    if (e != cudaSuccess) return cleanup(e, "serving slot");
    slot_layout(c, &sl);
    e = cudaMemset(sl.words, 0, 16);
    if (e != cudaSuccess) return cleanup(e, "serving slot");
  }
  cudaError_t e = device_malloc(&S->batch_mem, batch_bytes);
  for (int k = 0; e == cudaSuccess && k < kMaxBatches; ++k) {
    e = cudaStreamCreateWithPriority(&S->batches[k].stream, cudaStreamNonBlocking, lo);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->batches[k].done, cudaEventDisableTiming);
    S->batches[k].counter = reinterpret_cast<int*>(static_cast<char*>(S->batch_mem) + 256 * k);
  }
  if (e != cudaSuccess) return cleanup(e, "serving batch stream");
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
  if (n > S->cfg.max_gaussians) {
    set_error("a scene of %lld Gaussians exceeds the slots' %lld", (long long)n,
              (long long)S->cfg.max_gaussians);
    return TGS_ERR_CAPACITY;
  }
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
  out->regrown = 0;
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
      cudaFree(sl.mem);
      cudaFreeHost(sl.host);
    }
    cudaStreamDestroy(sl.stream);
    cudaEventDestroy(sl.done);
  }
  for (Batch& b : S->batches) {
    cudaEventDestroy(b.done);
    cudaStreamDestroy(b.stream);
  }
  if (drained) {
    cudaFree(S->batch_mem);
    for (auto& kv : S->scenes) cudaFree(kv.second.mem);
  }
  delete S;
  if (!drained)
    return set_error("frames still running after %d ms: their device memory was not freed",
                     kDrainLimitMs),
           TGS_ERR_TIMEOUT;
  return TGS_OK;
}

}  // extern "C"
