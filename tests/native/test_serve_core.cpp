// Host-side tests of the rendering service's scheduling core (no GPU): admission, pause, ticket
// lifecycle, bounded waits, request time-outs with a late completion, stop, statistics, and a fake
// executor into which failures are injected (an error status, a request that never completes).
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <thread>

#include "../../paper_2605_17855_gb300/csrc/serve_core.h"

using tgs::serve::Core;
using tgs::serve::Request;

static int g_failures = 0;
#define CHECK(cond)                                                   \
  do {                                                                \
    if (!(cond)) {                                                    \
      std::fprintf(stderr, "%s:%d: CHECK(%s)\n", __FILE__, __LINE__, #cond); \
      ++g_failures;                                                   \
    }                                                                 \
  } while (0)

static Request req(int scene, int w = 64, int h = 48) {
  Request r;
  r.scene = scene;
  r.camera.width = w;
  r.camera.height = h;
  return r;
}

static void test_admission_and_fifo() {
  Core c(2, 0);
  uint64_t t1 = 0, t2 = 0, t3 = 0;
  CHECK(c.submit(req(0), &t1) == TGS_OK);
  CHECK(c.submit(req(1), &t2) == TGS_OK);
  CHECK(c.submit(req(0), &t3) == TGS_ERR_BUSY);  // max_inflight reached
  CHECK(t1 != t2);
  CHECK(c.scene_refs(0) == 1 && c.scene_refs(1) == 1);
  Request r;
  CHECK(c.next(&r) && r.ticket == t1);  // submission order
  CHECK(c.next(&r) && r.ticket == t2);
  CHECK(!c.next(&r));
  // still admitted until released: a new submission is refused
  CHECK(c.submit(req(0), &t3) == TGS_ERR_BUSY);
  c.complete(t1, TGS_OK);
  c.release(req(0));
  CHECK(c.submit(req(0), &t3) == TGS_OK);
  tgs_serve_stats st;
  c.stats(&st);
  CHECK(st.submitted == 3 && st.rejected == 2 && st.completed == 1 && st.inflight == 2);
}

static void test_pause() {
  Core c(4, 0);
  c.set_paused(true);
  uint64_t t = 0;
  CHECK(c.submit(req(0), &t) == TGS_OK);  // admitted while paused
  Request r;
  CHECK(!c.next(&r));
  c.set_paused(false);
  CHECK(c.next(&r) && r.ticket == t);
}

static void test_ticket_lifecycle_and_wait() {
  Core c(4, 0);
  uint64_t t = 0;
  CHECK(c.submit(req(0), &t) == TGS_OK);
  int32_t done = -1;
  tgs_status res = -1;
  CHECK(c.poll(t, &done, &res) == TGS_OK && done == 0);
  // bounded wait on a request nobody completes
  const auto t0 = tgs::serve::Clock::now();
  CHECK(c.wait(t, 30, &res) == TGS_ERR_TIMEOUT);
  CHECK(tgs::serve::Clock::now() - t0 >= std::chrono::milliseconds(25));
  // completion from another thread wakes the waiter
  std::thread worker([&] {
    std::this_thread::sleep_for(std::chrono::milliseconds(20));
    c.complete(t, TGS_OK);
  });
  CHECK(c.wait(t, 5000, &res) == TGS_OK && res == TGS_OK);
  worker.join();
  CHECK(c.poll(t, &done, &res) == TGS_ERR_NOT_FOUND);  // released
  CHECK(c.wait(t, 10, &res) == TGS_ERR_NOT_FOUND);
  CHECK(c.poll(12345, &done, &res) == TGS_ERR_NOT_FOUND);
}

static void test_timeout_then_late_completion() {
  Core c(4, 10);  // request time-out 10 ms
  uint64_t t = 0;
  CHECK(c.submit(req(3), &t) == TGS_OK);
  Request r;
  CHECK(c.next(&r));
  CHECK(!c.expired(r, tgs::serve::Clock::now()));
  std::this_thread::sleep_for(std::chrono::milliseconds(15));
  CHECK(c.expired(r, tgs::serve::Clock::now()));
  c.complete(t, TGS_ERR_TIMEOUT);  // what the executor does: the slot stays busy
  CHECK(c.scene_refs(3) == 1);     // the GPU may still read the scene
  c.complete(t, TGS_OK);           // the late completion is ignored
  c.release(r);
  CHECK(c.scene_refs(3) == 0);
  tgs_status res = -1;
  int32_t done = 0;
  CHECK(c.poll(t, &done, &res) == TGS_OK && done == 1 && res == TGS_ERR_TIMEOUT);
  tgs_serve_stats st;
  c.stats(&st);
  CHECK(st.completed == 0 && st.failed == 1 && st.inflight == 0);
}

static void test_stop_drops_queue() {
  Core c(8, 0);
  uint64_t t1 = 0, t2 = 0;
  CHECK(c.submit(req(0), &t1) == TGS_OK);
  CHECK(c.submit(req(0), &t2) == TGS_OK);
  Request r;
  CHECK(c.next(&r));  // t1 is in a slot, t2 still queued
  std::atomic<int> woke{0};
  std::thread waiter([&] {
    tgs_status res = -1;
    if (c.wait(t2, 5000, &res) == TGS_OK && res == TGS_ERR_BUSY) woke = 1;
  });
  std::this_thread::sleep_for(std::chrono::milliseconds(10));
  c.stop();
  waiter.join();
  CHECK(woke == 1);
  CHECK(c.stopping());
  CHECK(!c.next(&r));
  uint64_t t3 = 0;
  CHECK(c.submit(req(0), &t3) == TGS_ERR_BUSY);
  CHECK(c.scene_refs(0) == 1);  // the request in the slot still holds its scene
  c.complete(t1, TGS_OK);
  c.release(r);
  tgs_serve_stats st;
  c.stats(&st);
  CHECK(st.inflight == 0);
}

static void test_statistics() {
  std::vector<float> v;
  for (int i = 1; i <= 100; ++i) v.push_back((float)(101 - i));
  CHECK(Core::percentile(v, 0.50) == 51.0);
  CHECK(Core::percentile(v, 0.99) == 100.0);
  Core c(1000, 0);
  for (int k = 0; k < 300; ++k) {
    uint64_t t = 0;
    const int w = (k % 3 == 0) ? 640 : 1280, h = (k % 3 == 0) ? 480 : 720;
    CHECK(c.submit(req(0, w, h), &t) == TGS_OK);
    Request r;
    CHECK(c.next(&r));
    c.complete(t, TGS_OK);
    c.release(r);
  }
  tgs_serve_stats st;
  c.stats(&st);
  CHECK(st.num_resolutions == 2);
  CHECK(st.res[0].width == 640 && st.res[0].height == 480 && st.res[0].completed == 100);
  CHECK(st.res[1].width == 1280 && st.res[1].completed == 200);
  CHECK(st.res[0].p50_ms <= st.res[0].p99_ms && st.res[0].mean_ms >= 0.0);
  CHECK(st.completed == 300 && st.frames_per_second > 0.0);
}

// A fake executor thread: takes requests like the CUDA worker, fails every third one with a CUDA
// error and never completes the one for scene 99 (a lost request). Clients see the errors, and a
// bounded wait on the lost ticket times out.
static void test_fake_executor_with_injected_faults() {
  Core c(64, 0);
  std::atomic<bool> quit{false};
  std::thread exec([&] {
    int k = 0;
    while (!quit) {
      Request r;
      if (!c.next(&r)) {
        c.wait_for_work(5);
        continue;
      }
      if (r.scene == 99) continue;  // dropped: neither completed nor released
      c.complete(r.ticket, (k++ % 3 == 2) ? TGS_ERR_CUDA : TGS_OK);
      c.release(r);
    }
  });
  std::vector<uint64_t> tickets;
  for (int i = 0; i < 30; ++i) {
    uint64_t t = 0;
    CHECK(c.submit(req(i % 2), &t) == TGS_OK);
    tickets.push_back(t);
  }
  uint64_t lost = 0;
  CHECK(c.submit(req(99), &lost) == TGS_OK);
  int ok = 0, cuda = 0;
  for (uint64_t t : tickets) {
    tgs_status res = -1;
    CHECK(c.wait(t, 5000, &res) == TGS_OK);
    ok += res == TGS_OK;
    cuda += res == TGS_ERR_CUDA;
  }
  CHECK(ok == 20 && cuda == 10);
  tgs_status res = -1;
  CHECK(c.wait(lost, 50, &res) == TGS_ERR_TIMEOUT);
  quit = true;
  exec.join();
  tgs_serve_stats st;
  c.stats(&st);
  CHECK(st.completed == 20 && st.failed == 10 && st.inflight == 1);
}

int main() {
  test_admission_and_fifo();
  test_pause();
  test_ticket_lifecycle_and_wait();
  test_timeout_then_late_completion();
  test_stop_drops_queue();
  test_statistics();
  test_fake_executor_with_injected_faults();
  if (g_failures) {
    std::fprintf(stderr, "%d check(s) failed\n", g_failures);
    return 1;
  }
  std::printf("serve core: all checks passed\n");
  return 0;
}
