// Host side of the rendering service (tgs_serve_*): admission, tickets, bounded waits and latency
// statistics. It uses no CUDA: the executor in serve.cu drives it from its worker thread, and it
// builds alone with a host C++17 compiler.
//
// A request is "admitted" from tgs_serve_submit until its slot is released by the executor (or it
// is dropped); admission is refused with TGS_ERR_BUSY beyond max_inflight. Its ticket "completes"
// once, with a status; a late second completion (the GPU work of a request that already timed
// out) is ignored. A completed ticket is released when poll or wait reports it.
#pragma once

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "../../include/tgs.h"

namespace tgs {
namespace serve {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  int32_t scene = -1;
  tgs_camera camera{};
  float* out_rgb = nullptr;
  float* out_T = nullptr;
  Clock::time_point submitted{};
};

class Core {
 public:
  static constexpr size_t kRing = 4096;  // latencies kept per resolution

  Core(int max_inflight, int request_timeout_ms)
      : max_inflight_(max_inflight), timeout_ms_(request_timeout_ms), t0_(Clock::now()) {}

  // ---- client side --------------------------------------------------------------------------
  tgs_status submit(Request r, uint64_t* ticket) {
    std::lock_guard<std::mutex> lock(mu_);
    if (stop_) return TGS_ERR_BUSY;
    if (inflight_ >= max_inflight_) {
      ++rejected_;
      return TGS_ERR_BUSY;
    }
    r.ticket = next_ticket_++;
    r.submitted = Clock::now();
    tickets_[r.ticket] = Ticket{TGS_OK, false, r.camera.width, r.camera.height, r.submitted};
    ++scene_refs_[r.scene];
    ++inflight_;
    ++submitted_;
    *ticket = r.ticket;
    queue_.push_back(r);
    cv_work_.notify_one();
    return TGS_OK;
  }

  tgs_status poll(uint64_t ticket, int32_t* done, tgs_status* result) {
    std::lock_guard<std::mutex> lock(mu_);
    auto it = tickets_.find(ticket);
    if (it == tickets_.end()) return TGS_ERR_NOT_FOUND;
    *done = it->second.done ? 1 : 0;
    if (it->second.done) {
      if (result) *result = it->second.status;
      tickets_.erase(it);
    }
    return TGS_OK;
  }

  tgs_status wait(uint64_t ticket, int32_t timeout_ms, tgs_status* result) {
    std::unique_lock<std::mutex> lock(mu_);
    auto it = tickets_.find(ticket);
    if (it == tickets_.end()) return TGS_ERR_NOT_FOUND;
    const auto deadline = Clock::now() + std::chrono::milliseconds(std::max(timeout_ms, 0));
    while (true) {
      it = tickets_.find(ticket);
      if (it == tickets_.end()) return TGS_ERR_NOT_FOUND;  // released by another thread
      if (it->second.done) break;
      if (cv_done_.wait_until(lock, deadline) == std::cv_status::timeout) {
        it = tickets_.find(ticket);
        if (it == tickets_.end()) return TGS_ERR_NOT_FOUND;
        if (!it->second.done) return TGS_ERR_TIMEOUT;
        break;
      }
    }
    if (result) *result = it->second.status;
    tickets_.erase(it);
    return TGS_OK;
  }

  void set_paused(bool paused) {
    std::lock_guard<std::mutex> lock(mu_);
    paused_ = paused;
    cv_work_.notify_all();
  }

  int64_t scene_refs(int32_t scene) const {
    std::lock_guard<std::mutex> lock(mu_);
    auto it = scene_refs_.find(scene);
    return it == scene_refs_.end() ? 0 : it->second;
  }

  void stats(tgs_serve_stats* out) const {
    std::lock_guard<std::mutex> lock(mu_);
    *out = tgs_serve_stats{};
    out->submitted = submitted_;
    out->rejected = rejected_;
    out->completed = completed_;
    out->failed = failed_;
    out->inflight = inflight_;
    out->seconds = std::chrono::duration<double>(Clock::now() - t0_).count();
    out->frames_per_second = out->seconds > 0 ? (double)completed_ / out->seconds : 0.0;
    out->num_resolutions = (int32_t)std::min(res_.size(), (size_t)TGS_SERVE_MAX_RESOLUTIONS);
    for (int k = 0; k < out->num_resolutions; ++k) {
      const Res& r = res_[k];
      tgs_serve_resolution_stats& o = out->res[k];
      o.width = r.w;
      o.height = r.h;
      o.completed = r.completed;
      std::vector<float> v(r.ring);
      if (v.empty()) continue;
      double sum = 0.0;
      for (float x : v) sum += x;
      o.mean_ms = sum / (double)v.size();
      o.p50_ms = percentile(v, 0.50);
      o.p99_ms = percentile(v, 0.99);
    }
  }

  // ---- executor side ------------------------------------------------------------------------
  // Pops the oldest queued request unless paused or stopping.
  bool next(Request* r) {
    std::lock_guard<std::mutex> lock(mu_);
    if (paused_ || stop_ || queue_.empty()) return false;
    *r = queue_.front();
    queue_.pop_front();
    return true;
  }

  // Blocks up to timeout_ms until a request can be popped or the core is stopping.
  void wait_for_work(int timeout_ms) {
    std::unique_lock<std::mutex> lock(mu_);
    cv_work_.wait_for(lock, std::chrono::milliseconds(timeout_ms),
                      [&] { return stop_ || (!paused_ && !queue_.empty()); });
  }

  // Completes a ticket (first call only) and records the latency of a successful request.
  void complete(uint64_t ticket, tgs_status status) {
    std::lock_guard<std::mutex> lock(mu_);
    auto it = tickets_.find(ticket);
    if (it == tickets_.end() || it->second.done) return;
    it->second.done = true;
    it->second.status = status;
    if (status == TGS_OK) {
      ++completed_;
      const float ms =
          std::chrono::duration<float, std::milli>(Clock::now() - it->second.submitted).count();
      Res& r = resolution(it->second.w, it->second.h);
      ++r.completed;
      if (r.ring.size() < kRing) {
        r.ring.push_back(ms);
      } else {
        r.ring[r.pos] = ms;
        r.pos = (r.pos + 1) % kRing;
      }
    } else {
      ++failed_;
    }
    cv_done_.notify_all();
  }

  // The request has left its slot (or was never placed): it no longer counts as admitted and no
  // longer holds its scene.
  void release(const Request& r) {
    std::lock_guard<std::mutex> lock(mu_);
    --inflight_;
    auto it = scene_refs_.find(r.scene);
    if (it != scene_refs_.end() && --it->second == 0) scene_refs_.erase(it);
  }

  bool expired(const Request& r, Clock::time_point now) const {
    return timeout_ms_ > 0 && now - r.submitted > std::chrono::milliseconds(timeout_ms_);
  }

  // Stops admission and dispatch; queued requests are dropped (completed with TGS_ERR_BUSY and
  // released). Wakes every waiter.
  void stop() {
    std::lock_guard<std::mutex> lock(mu_);
    stop_ = true;
    for (const Request& r : queue_) {
      auto it = tickets_.find(r.ticket);
      if (it != tickets_.end() && !it->second.done) {
        it->second.done = true;
        it->second.status = TGS_ERR_BUSY;
        ++failed_;
      }
      --inflight_;
      auto s = scene_refs_.find(r.scene);
      if (s != scene_refs_.end() && --s->second == 0) scene_refs_.erase(s);
    }
    queue_.clear();
    cv_work_.notify_all();
    cv_done_.notify_all();
  }

  bool stopping() const {
    std::lock_guard<std::mutex> lock(mu_);
    return stop_;
  }

 private:
  struct Ticket {
    tgs_status status;
    bool done;
    int32_t w, h;
    Clock::time_point submitted;
  };
  struct Res {
    int32_t w = 0, h = 0;
    int64_t completed = 0;
    std::vector<float> ring;
    size_t pos = 0;
  };

  Res& resolution(int32_t w, int32_t h) {
    for (Res& r : res_)
      if (r.w == w && r.h == h) return r;
    res_.push_back(Res{});
    res_.back().w = w;
    res_.back().h = h;
    return res_.back();
  }


 public:
  // Nearest-rank percentile of v (reorders v).
  static double percentile(std::vector<float>& v, double q) {
    size_t k = (size_t)(q * (double)v.size());
    if (k >= v.size()) k = v.size() - 1;
    std::nth_element(v.begin(), v.begin() + (ptrdiff_t)k, v.end());
    return v[k];
  }

 private:
  mutable std::mutex mu_;
  std::condition_variable cv_work_, cv_done_;
  std::deque<Request> queue_;
  std::unordered_map<uint64_t, Ticket> tickets_;
  std::unordered_map<int32_t, int64_t> scene_refs_;
  uint64_t next_ticket_ = 1;
  int max_inflight_;
  int timeout_ms_;
  int64_t inflight_ = 0;
  bool paused_ = false, stop_ = false;
  int64_t submitted_ = 0, rejected_ = 0, completed_ = 0, failed_ = 0;
  Clock::time_point t0_;
  std::vector<Res> res_;
};

}  // namespace serve
}  // namespace tgs
