// Internal helpers of the tgs library: error plumbing, PTX wrappers for mbarriers, tcgen05 tensor
// memory and MMA on sm_103a, and small numeric helpers. Not part of the ABI.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tgs.h"

namespace tgs {

// ---------------------------------------------------------------------------------------------
// Host-side error plumbing (implemented in abi.cu).
void set_error(const char* fmt, ...);
tgs_status cuda_status(cudaError_t e, const char* what);
// Device-side error word of the current device: a zero-initialized __device__ variable of the
// library (nothing is allocated); its address is looked up once per device.
int32_t* device_error_word();

#define TGS_CUDA(expr)                                              \
  do {                                                              \
    cudaError_t _e = (expr);                                        \
    if (_e != cudaSuccess) return ::tgs::cuda_status(_e, #expr);    \
  } while (0)

void note_launch();  // counts kernel launches (tgs_kernel_launch_count)
// The library's only ways to allocate memory (device, and pinned host); both are counted
// (tgs_allocation_count).
cudaError_t device_malloc(void** p, size_t bytes);
cudaError_t pinned_malloc(void** p, size_t bytes);

#define TGS_CHECK_LAUNCH(what)                                      \
  do {                                                              \
    ::tgs::note_launch();                                           \
    cudaError_t _e = cudaGetLastError();                            \
    if (_e != cudaSuccess) return ::tgs::cuda_status(_e, what);     \
  } while (0)

constexpr int kTile = TGS_TILE;

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Launchers implemented by the kernel translation units.
tgs_status launch_preprocess(const tgs_scene& s, const tgs_camera& cam, const tgs_projected& out,
                             cudaStream_t st);
size_t bin_sort_workspace_bytes(int64_t n, int64_t capacity, int GX, int GY);
// The word of a bin sort workspace that a call sets when one of its look-back waits ran out (n > 0).
int32_t* bin_sort_failed_word(void* ws, int64_t n, int64_t capacity, int GX, int GY);
// The limit of one look-back wait of the bin sort for calls launched after it; ns <= 0 restores the
// default. Returns the previous limit.
constexpr int64_t kDefaultLookbackLimitNs = 1000000000;  // 1 s
int64_t set_lookback_limit_ns(int64_t ns);
// err_word: the device word its bounded waits report to (NULL: the library's error word);
// overflow_word: optional device word set to 1 when the frame needs more entries than the capacity.
tgs_status launch_bin_sort(const tgs_projected& p, int64_t n, int width, int height, int gw, int gh,
                           bool membership, void* ws, size_t ws_bytes, const tgs_bins& bins,
                           cudaStream_t st, int32_t* err_word = nullptr,
                           int32_t* overflow_word = nullptr);
tgs_status launch_raster_fp32(const tgs_projected& p, const tgs_bins& b, int width, int height,
                              int gw, int gh, const tgs_raster_opts& o, float* out_rgb, float* out_T,
                              int32_t* n_contrib, cudaStream_t st);
tgs_status launch_raster_tc(const tgs_projected& p, const tgs_bins& b, int width, int height, int gw,
                            int gh, const tgs_raster_opts& o, float* out_rgb, float* out_T,
                            int32_t* n_contrib, cudaStream_t st);
tgs_status launch_raster_tc_bf16(const tgs_projected& p, const tgs_bins& b, int width, int height, int gw,
                            int gh, const tgs_raster_opts& o, float* out_rgb, float* out_T,
                            int32_t* n_contrib, cudaStream_t st);
// One frame of a batched tensor-core rasterization (tgs_rasterize_batch).
struct RasterFrame {
  const tgs_projected* p;
  const tgs_bins* b;
  int width, height;
  float* out_rgb;
  float* out_T;
  const int32_t* ready;
  int32_t ready_value;
  int32_t* status;
  int32_t* done;
  int32_t done_value;
};
// share_div > 1 limits the persistent grid to 1/share_div of the GPU's resident CTA slots, so
// that another launch can run beside it.
tgs_status launch_raster_tc_batch(const RasterFrame* frames, int count, int gw, int gh,
                                  const tgs_raster_opts& o, int* next_item, uint64_t wait_ns,
                                  cudaStream_t st, int share_div = 1);
tgs_status launch_raster_tc_batch_bf16(const RasterFrame* frames, int count, int gw, int gh,
                                       const tgs_raster_opts& o, int* next_item, uint64_t wait_ns,
                                       cudaStream_t st, int share_div);
tgs_status launch_raster_backward(const tgs_projected& p, int64_t n, const tgs_bins& b, int width,
                                  int height, int gw, int gh, const tgs_raster_opts& o,
                                  const float* out_T, const int32_t* n_contrib, const float* grad_rgb,
                                  float* g_mean2d, float* g_conic_opacity, float* g_rgb,
                                  cudaStream_t st);

// ---------------------------------------------------------------------------------------------
// Device helpers.

// Blend constants of Section 2 (pruning threshold, clamp, termination threshold).
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kLog2e = 1.4426950408889634f;

// Hardware base-2 exponential (PTX ex2.approx.ftz.f32).
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// Hardware base-2 logarithm (PTX lg2.approx.ftz.f32).
__device__ __forceinline__ float lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Upper Cholesky factor L = [[l11, l12], [0, l22]] of a conic [[a, b], [b, c]] (conic = L^T L),
// computed once per list entry. The determinant a c - b^2 uses Kahan's compensated 2x2 scheme
// (one FMA recovers the rounding error of b^2), so thin splats, whose determinant is a small
// difference of large products, keep full relative accuracy.
__device__ __forceinline__ float3 conic_factor(float a, float b, float c) {
  const float w = __fmul_rn(b, b);
  const float e = __fmaf_rn(-b, b, w);  // w - b*b, exactly
  const float det = __fadd_rn(__fmaf_rn(a, c, -w), e);
  const float l11 = sqrtf(a);
  return make_float3(l11, __fdiv_rn(b, l11), sqrtf(fmaxf(__fdiv_rn(det, a), 0.f)));
}

// Power of Eq. power, -1/2 d^T conic d, evaluated as -1/2 |L d|^2: a sum of two squares, so it is
// never positive and does not suffer the cancellation of the expanded form of
// Eq. tensorgs_power_scalar when d is large along a thin splat. Fixed operation order: the FP32
// forward, the backward replay and the scalar rows of the tensor path agree bit for bit.
__device__ __forceinline__ float power_fp32(float3 L, float dx, float dy) {
  const float u = __fmaf_rn(L.x, dx, __fmul_rn(L.y, dy));
  const float v = __fmul_rn(L.z, dy);
  return __fmul_rn(-0.5f, __fmaf_rn(u, u, __fmul_rn(v, v)));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier -----------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// As mbar_try_wait, with a hint of how long (ns) the thread may stay suspended waiting for the
// phase before the call returns false; a suspended warp issues no instructions.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t* bar, uint32_t parity,
                                                   uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
// Non-blocking test of an mbarrier phase.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Invalidates an mbarrier (no operation may be pending on it), so its memory can be re-initialized.
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Arrive `count` times at once.
__device__ __forceinline__ void mbar_arrive_n(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
// Longest suspension of one try-wait inside the bounded waits below; the abort flag and the time
// limit are checked between them.
constexpr uint32_t kSuspendHintNs = 20000;
// The same for waits that a stop flag can end: the flag is no barrier event, so a suspended waiter
// sees it only when the hint expires.
constexpr uint32_t kStopHintNs = 1000;
// Bounded wait: gives up after `limit_ns` (or when *abort is set) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  volatile int* abort, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait_hint(bar, parity, kSuspendHintNs)) return true;
    if (*abort) return false;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// Bounded wait that also ends when *stop is set: 0 = phase complete, 1 = stopped, 2 = timed out
// or aborted.
__device__ __forceinline__ int mbar_wait_or_stop(uint64_t* bar, uint32_t parity, volatile int* stop,
                                                 volatile int* abort, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return 0;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait_hint(bar, parity, kStopHintNs)) return 0;
    if (*stop) return 1;
    if (*abort) return 2;
    if (globaltimer_ns() - t0 > limit_ns) return 2;
  }
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbarrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// ---- tcgen05: tensor memory ---------------------------------------------------------------
// Allocation is done by one whole warp; the TMEM address is written to shared memory.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_addr(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor for tcgen05.mma, no swizzle, K-major canonical layout:
// core matrices of 8 rows x 16 bytes (rows 16 B apart); `lbo` = byte distance between the two core
// matrices adjacent along K, `sbo` = byte distance between 8-row groups along M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  // base offset 0, absolute LBO mode 0, layout type 0 (no swizzle)
  return d;
}

// Instruction descriptor of tcgen05.mma.kind::f16 with FP32 accumulation, both operands K-major.
// ab_bf16 selects BF16 (else FP16) for A and B.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, bool ab_bf16) {
  return (1u << 4)                              // D format: F32
         | ((ab_bf16 ? 1u : 0u) << 7)           // A format
         | ((ab_bf16 ? 1u : 0u) << 10)          // B format
         | ((uint32_t)(N >> 3) << 17)           // N / 8
         | ((uint32_t)(M >> 4) << 24);          // M / 16
}

// D[tmem] (=|+=) A[smem] * B[smem]^T, issued by a single thread.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on `bar` once all tcgen05 operations previously issued by this thread complete.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

// Tensor-memory loads, shape 32x32b (lane of the warp = TMEM lane 32 * (warp % 4) + laneid),
// 8 consecutive 32-bit columns at each of two addresses, without waiting. The registers must not be
// read before tmem_wait_ld(r), which names them as operands so that every use stays after it.
__device__ __forceinline__ void tmem_ld8x2_async(uint32_t ta, uint32_t tb, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%16];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%17];"
      : "=r"(r[0]),"=r"(r[1]),"=r"(r[2]),"=r"(r[3]),"=r"(r[4]),"=r"(r[5]),"=r"(r[6]),"=r"(r[7]),"=r"(r[8]),"=r"(r[9]),"=r"(r[10]),"=r"(r[11]),"=r"(r[12]),"=r"(r[13]),"=r"(r[14]),"=r"(r[15])
      : "r"(ta), "r"(tb)
      : "memory");
}
// One tensor-memory load of 8 consecutive 32-bit columns (shape 32x32b), without waiting; read the
// registers only after tmem_wait_ld8(r).
__device__ __forceinline__ void tmem_ld8_async(uint32_t ta, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]),"=r"(r[1]),"=r"(r[2]),"=r"(r[3]),"=r"(r[4]),"=r"(r[5]),"=r"(r[6]),"=r"(r[7])
               : "r"(ta)
               : "memory");
}
// Two tensor-memory loads of 4 consecutive columns each (pixel blocks at ta and tb) into r[0..3] and
// r[4..7], without waiting; read them only after tmem_wait_ld8(r).
__device__ __forceinline__ void tmem_ld4x2_async(uint32_t ta, uint32_t tb, uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%8];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4,%5,%6,%7}, [%9];"
      : "=r"(r[0]),"=r"(r[1]),"=r"(r[2]),"=r"(r[3]),"=r"(r[4]),"=r"(r[5]),"=r"(r[6]),"=r"(r[7])
      : "r"(ta), "r"(tb)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld8(uint32_t (&r)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]),"+r"(r[1]),"+r"(r[2]),"+r"(r[3]),"+r"(r[4]),"+r"(r[5]),"+r"(r[6]),"+r"(r[7]) : : "memory");
}
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]),"+r"(r[1]),"+r"(r[2]),"+r"(r[3]),"+r"(r[4]),"+r"(r[5]),"+r"(r[6]),"+r"(r[7]),"+r"(r[8]),"+r"(r[9]),"+r"(r[10]),"+r"(r[11]),"+r"(r[12]),"+r"(r[13]),"+r"(r[14]),"+r"(r[15]) : : "memory");
}

}  // namespace tgs
