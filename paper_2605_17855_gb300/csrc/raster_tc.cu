// Grouped tensor-core rasterizer (Section 4.2 "Tensorizing the power computation" and Section 4.4.2
// "Grouped rasterization"; Algorithm 1, the per-group CTA loop), written for sm_103a with tcgen05.
//
// One CTA per tile group. The group's depth-sorted list is consumed in chunks of NB entries:
//   * producer warps (several, on interleaved chunks): gather the chunk's Gaussians (mean, conic,
//     opacity, colour, mask) and, for
//     every member tile whose mask bit is set, writes the Gaussian's coefficient row of the power
//     expansion about that tile's centre (o_x, o_y) = (16 tx + 8, 16 ty + 8). With pixel offsets
//     (x, y) = (px - o_x, py - o_y) and (mx, my) = mu' - o:
//        log2(o) + log2(e) * power = q . [x^2, xy, y^2, x, y, 1]
//        q = log2(e) * (-a/2, -b, -c/2, a mx + b my, b mx + c my, -(a mx^2 + 2 b mx my + c my^2)/2)
//            + (0, 0, 0, 0, 0, log2 o)
//     This is the expansion of Eq. tensorgs_power_scalar about a common origin, which makes the
//     power a true matrix product (the Q Phi of Section 4.2.2 with the per-pixel terms separated
//     from the per-Gaussian ones). q is split into FP16 hi + lo and the K dimension holds
//     [hi(6), lo(6), 0, 0, 0, 0] against features [f(6), f(6), 0, 0, 0, 0]: the zero padding of
//     Section 4.2.3 (exact), with the padding slots used for the lo half. |x|, |y| <= 8, so every
//     feature is an exact FP16 integer. Rows whose FP16 error bound is too large take a scalar
//     FP32 path in the epilogue instead.
//   * MMA thread: per tile, D[128 px x NB] = A_h[128 x 16] * B_t[NB x 16]^T with
//     tcgen05.mma.cta_group::1.kind::f16 (M = 128, N = NB, K = 16), FP32 accumulators in tensor
//     memory, double-buffered; completion signalled through tcgen05.commit on mbarriers.
//   * epilogue warpgroups (one per tile of a round): each thread owns one TMEM lane = one pixel in
//     each of the tile's two 128-pixel M blocks, loads its NB exponents with tcgen05.ld and runs
//     the front-to-back blend of Section 2 in FP32 (skip if alpha < 1/255 tested in the log2
//     domain before the exp, alpha = min(0.99, 2^D), stop when T' < 1e-4 without blending).
// The chunk is loaded from global memory once per group and reused by all member tiles
// (the cross-tile reuse of Section 4.4.2); a tile ignores entries whose mask bit is clear, which
// keeps each tile's front-to-back order (Section 4.4.2, numerical equivalence).
// Termination: before each chunk the MMA thread checks whether every epilogue warp has finished
// all its pixels (T < 1e-4 or end of list); if so it stops issuing, raises a stop flag for the
// producers and signals the epilogue the index of the last job.
// Every wait on an mbarrier is bounded (2 s); on expiry the CTA records TGS_ERR_TIMEOUT in the
// device error word, drains its MMAs, frees its tensor memory and exits.
#include <algorithm>

#include "tgs_internal.cuh"

namespace tgs {
namespace {

constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr float kL255 = -7.994353436858858f;  // log2(1/255)
constexpr float kLog2AlphaMax = -0.014499569695115089f;  // log2(0.99)
// Rows whose FP16 hi/lo error bound 2^-22 * sum_k |q_k| max|f_k| exceeds this (in log2 units)
// are evaluated by the scalar FP32 path.
constexpr float kMaxWeightedCoef = 4096.0f;
constexpr int kLBO = 128;  // bytes between the two K core matrices of an 8-row group
constexpr int kSBO = 256;  // bytes between 8-row groups

template <int GW, int GH, int NWG, int NB, int NPROD>
struct Cfg {
  static constexpr int kTiles = GW * GH;
  static constexpr int kRounds = kTiles / NWG;
  static_assert(kTiles % NWG == 0, "tiles must split evenly over warpgroups");
  static constexpr int kEpiWarps = 4 * NWG;
  static constexpr int kProdWarp0 = kEpiWarps;
  static constexpr int kMmaWarp = kEpiWarps + NPROD;
  static constexpr int kThreads = 32 * (kMmaWarp + 1);
  static constexpr int kSlots = 2 * NPROD;  // each producer owns the slots s with s % NPROD == p
  static constexpr int kStageCols = NWG * 2 * NB;
  static constexpr int kTmemCols = 2 * kStageCols;
  static_assert(kTmemCols == 32 || kTmemCols == 64 || kTmemCols == 128 || kTmemCols == 256 ||
                    kTmemCols == 512,
                "TMEM allocation must be a power of two in [32, 512]");
  static_assert(NB == 32, "the producer maps one list entry to one lane of its warp");
};

template <int TILES, int NB>
struct __align__(16) Slot {
  uint8_t B[TILES][NB * 32];  // K-major canonical, no swizzle: (row/8)*256 + (k/8)*128 + (row%8)*16
  float4 rgbc[NB];            // colour, cap = min(log2 o, log2 0.99)
  float4 sp0[NB];             // mu'x, mu'y, l11, l12  (scalar rows; Cholesky factor of the conic)
  float2 sp1[NB];             // l22, log2 o
  uint32_t tbits[TILES];      // bit j: entry j is used by tile t
  uint32_t sbits[TILES];      // bit j: entry j uses the scalar path for tile t
  int32_t base;               // list position of entry 0 relative to the group start
};

template <int TILES, int NB, int SLOTS>
struct __align__(1024) Smem {
  uint8_t A[2][4096];  // two 128-pixel M blocks of the tile feature operand
  Slot<TILES, NB> slot[SLOTS];
  uint64_t full[SLOTS], empty[SLOTS], tfull[2], tempty[2], drain;
  uint32_t tmem_base;
  int abort;       // a bounded wait expired somewhere in the CTA
  int stop;        // the MMA thread stopped issuing: producers quit
  int end_job;     // index of the job whose tfull phase signals the end (-1 until known)
  int done_warps;  // epilogue warps whose pixels have all finished
};

// Pixel of TMEM lane m (0..127) of M block h inside a 16x16 tile: warp quarters are 8x4 pixels.
__device__ __forceinline__ void lane_pixel(int h, int m, int& lx, int& ly) {
  const int bi = h * 4 + (m >> 5), l = m & 31;
  lx = (bi & 1) * 8 + (l & 7);
  ly = (bi >> 1) * 4 + (l >> 3);
}

__device__ __forceinline__ uint32_t pack_h2(float lo_elem, float hi_elem) {
  const __half2 h = __floats2half2_rn(lo_elem, hi_elem);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ void record_abort(int* abort_flag, int32_t* err) {
  *reinterpret_cast<volatile int*>(abort_flag) = 1;
  if (err) atomicExch(err, TGS_ERR_TIMEOUT);
}

struct PixState {
  float T, r, g, b;
  int last;
  bool done;
};

template <bool COUNT>
__device__ __forceinline__ void blend_step(float e, const float4& rc, PixState& s, int pos,
                                           unsigned long long& passing) {
  const float d = fminf(e, rc.w);
  if (!s.done && d >= kL255) {
    if (COUNT) ++passing;
    const float a = ex2(d);
    const float Tn = fmaf(-s.T, a, s.T);
    if (Tn < kTMin) {
      s.done = true;
    } else {
      const float w = a * s.T;
      s.r = fmaf(w, rc.x, s.r);
      s.g = fmaf(w, rc.y, s.g);
      s.b = fmaf(w, rc.z, s.b);
      s.T = Tn;
      s.last = pos;
    }
  }
}

__device__ __forceinline__ float scalar_exponent(float px, float py, const float4& p0,
                                                 const float2& p1) {
  const float dx = __fsub_rn(px, p0.x), dy = __fsub_rn(py, p0.y);
  return fmaf(power_fp32(make_float3(p0.z, p0.w, p1.x), dx, dy), kLog2e, p1.y);
}

template <int GW, int GH, int NWG, int NB, int NPROD, bool COUNT>
__global__ void __launch_bounds__(Cfg<GW, GH, NWG, NB, NPROD>::kThreads, 1)
    k_raster_tc(const uint32_t* __restrict__ ranges, const uint32_t* __restrict__ vals,
                const uint16_t* __restrict__ masks, const float2* __restrict__ mean2d,
                const float4* __restrict__ conic_opacity, const float* __restrict__ rgb, int width,
                int height, int GX, float3 bg, float* __restrict__ out_rgb,
                float* __restrict__ out_T, int* __restrict__ n_contrib,
                unsigned long long* __restrict__ counters, int32_t* __restrict__ err) {
  using C = Cfg<GW, GH, NWG, NB, NPROD>;
  constexpr int TILES = C::kTiles;
  constexpr int SLOTS = C::kSlots;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  auto& S = *reinterpret_cast<Smem<TILES, NB, SLOTS>*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gid = blockIdx.x;
  const int gx = gid % GX, gy = gid / GX;

  // ---- set-up: feature operand A, barriers, tensor memory -------------------------------------
  for (int m = threadIdx.x; m < 256; m += blockDim.x) {
    const int h = m >> 7, row = m & 127;
    int lx, ly;
    lane_pixel(h, row, lx, ly);
    const float x = (float)(lx - 8), y = (float)(ly - 8);
    const float f[6] = {x * x, x * y, y * y, x, y, 1.f};
    uint4 c0, c1;
    c0.x = pack_h2(f[0], f[1]); c0.y = pack_h2(f[2], f[3]); c0.z = pack_h2(f[4], f[5]);
    c0.w = pack_h2(f[0], f[1]);
    c1.x = pack_h2(f[2], f[3]); c1.y = pack_h2(f[4], f[5]); c1.z = 0u; c1.w = 0u;
    uint8_t* rowp = &S.A[h][(row >> 3) * kSBO + (row & 7) * 16];
    *reinterpret_cast<uint4*>(rowp) = c0;
    *reinterpret_cast<uint4*>(rowp + kLBO) = c1;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < SLOTS; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], C::kEpiWarps + 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&S.tfull[s], 1);
      mbar_init(&S.tempty[s], C::kEpiWarps);
    }
    mbar_init(&S.drain, 1);
    S.abort = 0;
    S.stop = 0;
    S.end_job = -1;
    S.done_warps = 0;
    fence_mbarrier_init();
  }
  if (warp == C::kMmaWarp) {
    tmem_alloc(&S.tmem_base, C::kTmemCols);
    tmem_relinquish();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;
  volatile int* abort_flag = &S.abort;
  volatile int* stop_flag = &S.stop;

  const uint32_t list_start = ranges[2 * gid], list_end = ranges[2 * gid + 1];
  const int nchunks = (int)((list_end - list_start + NB - 1) / NB);

  if (warp >= C::kProdWarp0 && warp < C::kMmaWarp) {
    // ---- producers: gather + coefficient rows, chunks c = p, p + NPROD, ... ------------------
    for (int c = warp - C::kProdWarp0; c < nchunks; c += NPROD) {
      const int s = c % SLOTS;
      const int w = mbar_wait_or_stop(&S.empty[s], ((c / SLOTS) & 1) ^ 1, stop_flag, abort_flag,
                                      kWaitLimitNs);
      const int wmax = __reduce_max_sync(0xffffffffu, w);
      if (wmax == 1 && __reduce_min_sync(0xffffffffu, w) >= 1) break;  // stopped: not an error
      if (wmax != 0) {
        if (wmax == 2) record_abort(&S.abort, err);
        break;
      }
      auto& sl = S.slot[s];
      const uint32_t e = list_start + (uint32_t)c * NB + lane;
      const bool valid = e < list_end;
      float2 mu = make_float2(0.f, 0.f);
      float4 co = make_float4(0.f, 0.f, 0.f, 1.f);
      float3 col = make_float3(0.f, 0.f, 0.f);
      uint32_t msk = 0;
      if (valid) {
        const uint32_t i = vals[e];
        msk = masks[e];
        mu = mean2d[i];
        co = conic_opacity[i];
        col = make_float3(rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2]);
      }
      const float lo2 = lg2(co.w);
      const float3 Lc = valid ? conic_factor(co.x, co.y, co.z) : make_float3(0.f, 0.f, 0.f);
      sl.rgbc[lane] = make_float4(col.x, col.y, col.z, fminf(lo2, kLog2AlphaMax));
      sl.sp0[lane] = make_float4(mu.x, mu.y, Lc.x, Lc.y);
      sl.sp1[lane] = make_float2(Lc.z, lo2);
#pragma unroll
      for (int t = 0; t < TILES; ++t) {
        const int tx = gx * GW + (t % GW), ty = gy * GH + (t / GW);
        const bool active = valid && ((msk >> t) & 1u);
        bool scalar = false;
        uint4 r0 = make_uint4(0u, 0u, 0u, 0u), r1 = make_uint4(0u, 0u, 0u, 0u);
        if (active) {
          const float mx = mu.x - (float)(tx * kTile + 8), my = mu.y - (float)(ty * kTile + 8);
          // (u, v) = L m: the linear and constant terms are formed from it (conic m = L^T L m and
          // m^T conic m = u^2 + v^2), which avoids the cancellation of the expanded products when
          // the tile is far from the centre of a thin splat
          const float u = fmaf(Lc.x, mx, Lc.y * my), v = Lc.z * my;
          float q[6];
          q[0] = -0.5f * co.x * kLog2e;
          q[1] = -co.y * kLog2e;
          q[2] = -0.5f * co.z * kLog2e;
          q[3] = Lc.x * u * kLog2e;
          q[4] = fmaf(Lc.y, u, Lc.z * v) * kLog2e;
          q[5] = fmaf(-0.5f * kLog2e, fmaf(u, u, v * v), lo2);
          const float wsum = 64.f * (fabsf(q[0]) + fabsf(q[1]) + fabsf(q[2])) +
                             8.f * (fabsf(q[3]) + fabsf(q[4])) + fabsf(q[5]);
          scalar = !(wsum <= kMaxWeightedCoef);
          if (!scalar) {
            float hi[6], lo[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
              hi[k] = __half2float(__float2half_rn(q[k]));
              lo[k] = q[k] - hi[k];
            }
            r0.x = pack_h2(hi[0], hi[1]); r0.y = pack_h2(hi[2], hi[3]);
            r0.z = pack_h2(hi[4], hi[5]); r0.w = pack_h2(lo[0], lo[1]);
            r1.x = pack_h2(lo[2], lo[3]); r1.y = pack_h2(lo[4], lo[5]);
          }
        }
        uint8_t* rowp = &sl.B[t][(lane >> 3) * kSBO + (lane & 7) * 16];
        *reinterpret_cast<uint4*>(rowp) = r0;
        *reinterpret_cast<uint4*>(rowp + kLBO) = r1;
        const uint32_t tb = __ballot_sync(0xffffffffu, active);
        const uint32_t sb = __ballot_sync(0xffffffffu, active && scalar);
        if (lane == 0) {
          sl.tbits[t] = tb;
          sl.sbits[t] = sb;
        }
      }
      if (lane == 0) sl.base = c * NB;
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.full[s]);
    }
  } else if (warp == C::kMmaWarp) {
    // ---- MMA issuer ---------------------------------------------------------------------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(128, NB, false);
      const uint64_t adesc0 = smem_desc(smem_addr(&S.A[0][0]), kLBO, kSBO);
      const uint64_t adesc1 = smem_desc(smem_addr(&S.A[1][0]), kLBO, kSBO);
      int job = 0;
      bool failed = false;
      for (int c = 0; c < nchunks && !failed; ++c) {
        // every epilogue warp has finished all its pixels: no more work for this group
        if (*reinterpret_cast<volatile int*>(&S.done_warps) >= C::kEpiWarps) break;
        const int s = c % SLOTS;
        if (!mbar_wait_bounded(&S.full[s], (c / SLOTS) & 1, abort_flag, kWaitLimitNs)) {
          failed = true;
          break;
        }
        auto& sl = S.slot[s];
        for (int r = 0; r < C::kRounds; ++r, ++job) {
          const int st = job & 1;
          if (!mbar_wait_bounded(&S.tempty[st], ((job >> 1) & 1) ^ 1, abort_flag, kWaitLimitNs)) {
            failed = true;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int g = 0; g < NWG; ++g) {
            const int t = g + NWG * r;
            if (sl.tbits[t] == 0u) continue;
            const uint64_t bdesc = smem_desc(smem_addr(&sl.B[t][0]), kLBO, kSBO);
            const uint32_t col = (uint32_t)(st * C::kStageCols + (2 * g) * NB);
            mma_f16(tmem + col, adesc0, bdesc, idesc, 0u);
            mma_f16(tmem + col + NB, adesc1, bdesc, idesc, 0u);
          }
          mma_commit(&S.tfull[st]);
        }
        if (!failed) mma_commit(&S.empty[s]);
      }
      *stop_flag = 1;
      if (failed) {
        record_abort(&S.abort, err);
      } else {
        // end signal: complete the next tfull phase with a plain arrive after publishing its index
        const int st = job & 1;
        if (mbar_wait_bounded(&S.tempty[st], ((job >> 1) & 1) ^ 1, abort_flag, kWaitLimitNs)) {
          *reinterpret_cast<volatile int*>(&S.end_job) = job;
          mbar_arrive(&S.tfull[st]);
        } else {
          record_abort(&S.abort, err);
        }
      }
      // drain: all MMAs issued by this thread have completed before tensor memory is freed
      mma_commit(&S.drain);
      if (!mbar_wait_bounded(&S.drain, 0, abort_flag, kWaitLimitNs)) record_abort(&S.abort, err);
    }
    __syncwarp();
  } else {
    // ---- epilogue warpgroups ------------------------------------------------------------------
    const int wg = warp >> 2, quarter = warp & 3;
    int px[C::kRounds][2], py[C::kRounds][2];
    PixState ps[C::kRounds][2];
    bool wdone[C::kRounds];
#pragma unroll
    for (int r = 0; r < C::kRounds; ++r) {
      const int t = wg + NWG * r;
      const int tx = gx * GW + (t % GW), ty = gy * GH + (t / GW);
      bool all = true;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int lx, ly;
        lane_pixel(h, quarter * 32 + lane, lx, ly);
        px[r][h] = tx * kTile + lx;
        py[r][h] = ty * kTile + ly;
        const bool inside = px[r][h] < width && py[r][h] < height;
        ps[r][h] = PixState{1.f, 0.f, 0.f, 0.f, 0, !inside};
        all &= !inside;
      }
      wdone[r] = __all_sync(0xffffffffu, all);
    }
    bool counted_done = false;
    unsigned long long evaluated = 0, passing = 0;
    int job = 0;
    bool finished = false;
    for (int c = 0; !finished; ++c) {
      const int s = c % SLOTS;
#pragma unroll
      for (int r = 0; r < C::kRounds; ++r) {
        const int st = job & 1;
        bool ok = mbar_wait_bounded(&S.tfull[st], (job >> 1) & 1, abort_flag, kWaitLimitNs);
        if (!__all_sync(0xffffffffu, ok)) { record_abort(&S.abort, err); finished = true; break; }
        if (__shfl_sync(0xffffffffu, *reinterpret_cast<volatile int*>(&S.end_job), 0) == job) {
          finished = true;
          break;
        }
        if (r == 0) {
          // the slot's producer writes (colours, masks) are complete: the MMA thread waited on
          // the same phase before issuing this job
          ok = mbar_wait_bounded(&S.full[s], (c / SLOTS) & 1, abort_flag, kWaitLimitNs);
          if (!__all_sync(0xffffffffu, ok)) { record_abort(&S.abort, err); finished = true; break; }
        }
        ++job;
        tc_fence_after();
        auto& sl = S.slot[s];
        const int t = wg + NWG * r;
        const uint32_t tb = sl.tbits[t];
        const bool work = tb != 0u && !wdone[r];
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) +
                               (uint32_t)(st * C::kStageCols + (2 * wg) * NB);
        if (work) {
          const uint32_t sb = sl.sbits[t];
          const int base = sl.base;
          // NB/16 halves of 16 columns; the stage is released after the last load
#pragma unroll
          for (int half = 0; half < NB / 16; ++half) {
            float d0[16], d1[16];
            __syncwarp();  // tcgen05.ld is warp-collective: reconverge after the blend branches
            tmem_ld_2x16(taddr + half * 16, taddr + NB + half * 16, d0, d1);
            if (half == NB / 16 - 1) {
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&S.tempty[st]);
            }
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
              const int j = half * 16 + jj;
              if (!((tb >> j) & 1u)) continue;
              const float4 rc = sl.rgbc[j];
              float e0 = d0[jj], e1 = d1[jj];
              if ((sb >> j) & 1u) {
                const float4 p0 = sl.sp0[j];
                const float2 p1 = sl.sp1[j];
                e0 = scalar_exponent((float)px[r][0], (float)py[r][0], p0, p1);
                e1 = scalar_exponent((float)px[r][1], (float)py[r][1], p0, p1);
              }
              if (COUNT) evaluated += (!ps[r][0].done) + (!ps[r][1].done);
              blend_step<COUNT>(e0, rc, ps[r][0], base + j + 1, passing);
              blend_step<COUNT>(e1, rc, ps[r][1], base + j + 1, passing);
            }
          }
          wdone[r] = __all_sync(0xffffffffu, ps[r][0].done && ps[r][1].done);
        } else {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&S.tempty[st]);
        }
        if (r == C::kRounds - 1) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&S.empty[s]);
        }
      }
      if (!finished && !counted_done) {
        bool all = true;
#pragma unroll
        for (int r = 0; r < C::kRounds; ++r) all &= wdone[r];
        if (all) {
          counted_done = true;
          if (lane == 0) atomicAdd(&S.done_warps, 1);
        }
      }
    }
    // ---- outputs ------------------------------------------------------------------------------
    const size_t HW = (size_t)width * height;
#pragma unroll
    for (int r = 0; r < C::kRounds; ++r)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (px[r][h] >= width || py[r][h] >= height) continue;
        const size_t p = (size_t)py[r][h] * width + px[r][h];
        const PixState& q = ps[r][h];
        out_rgb[p] = q.r + q.T * bg.x;
        out_rgb[HW + p] = q.g + q.T * bg.y;
        out_rgb[2 * HW + p] = q.b + q.T * bg.z;
        out_T[p] = q.T;
        if (n_contrib) n_contrib[p] = q.last;
      }
    if (COUNT) {
      for (int o = 16; o > 0; o >>= 1) {
        evaluated += __shfl_xor_sync(0xffffffffu, evaluated, o);
        passing += __shfl_xor_sync(0xffffffffu, passing, o);
      }
      if (lane == 0) {
        if (evaluated) atomicAdd(counters, evaluated);
        if (passing) atomicAdd(counters + 1, passing);
      }
    }
  }

  // ---- teardown -----------------------------------------------------------------------------
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == C::kMmaWarp) tmem_dealloc(tmem, C::kTmemCols);
}

template <int GW, int GH, int NWG, int NB, int NPROD>
tgs_status launch_cfg(const tgs_projected& p, const tgs_bins& b, int width, int height,
                      const tgs_raster_opts& o, float* out_rgb, float* out_T, int32_t* n_contrib,
                      cudaStream_t st) {
  using Cf = Cfg<GW, GH, NWG, NB, NPROD>;
  using Sm = Smem<GW * GH, NB, Cf::kSlots>;
  const int TX = div_up(width, kTile), TY = div_up(height, kTile);
  const int GX = div_up(TX, GW), GY = div_up(TY, GH);
  // Limit residency so that co-resident CTAs never wait on each other's tensor memory:
  // at most 512 / kTmemCols CTAs per SM.
  int dev = 0, smem_sm = 0;
  TGS_CUDA(cudaGetDevice(&dev));
  TGS_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  const int max_ctas = 512 / Cf::kTmemCols;
  size_t smem = sizeof(Sm) + 1024;  // + alignment slack
  const size_t floor_bytes = (size_t)smem_sm / (max_ctas + 1) - 1024 + 16;
  smem = std::max(smem, floor_bytes);
  const bool count = o.counters != nullptr;
  auto* m2 = reinterpret_cast<const float2*>(p.mean2d);
  auto* co = reinterpret_cast<const float4*>(p.conic_opacity);
  auto* cnt = reinterpret_cast<unsigned long long*>(o.counters);
  const float3 bg = make_float3(o.bg[0], o.bg[1], o.bg[2]);
  int32_t* err = device_error_word();
  if (count) {
    auto* k = k_raster_tc<GW, GH, NWG, NB, NPROD, true>;
    TGS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<GX * GY, Cf::kThreads, smem, st>>>(b.ranges, b.vals, b.masks, m2, co, p.rgb, width, height, GX,
                                           bg, out_rgb, out_T, n_contrib, cnt, err);
  } else {
    auto* k = k_raster_tc<GW, GH, NWG, NB, NPROD, false>;
    TGS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<GX * GY, Cf::kThreads, smem, st>>>(b.ranges, b.vals, b.masks, m2, co, p.rgb, width, height, GX,
                                           bg, out_rgb, out_T, n_contrib, cnt, err);
  }
  TGS_CHECK_LAUNCH("k_raster_tc");
  return TGS_OK;
}

}  // namespace

tgs_status launch_raster_tc(const tgs_projected& p, const tgs_bins& b, int width, int height, int gw,
                            int gh, const tgs_raster_opts& o, float* out_rgb, float* out_T,
                            int32_t* n_contrib, cudaStream_t st) {
  if (((uintptr_t)p.mean2d & 7) || ((uintptr_t)p.conic_opacity & 15))
    return set_error("mean2d needs 8-byte and conic_opacity 16-byte alignment"), TGS_ERR_INVALID_ARGUMENT;
  if (gw == 1 && gh == 1) return launch_cfg<1, 1, 1, 32, 2>(p, b, width, height, o, out_rgb, out_T, n_contrib, st);
  if (gw == 2 && gh == 2) return launch_cfg<2, 2, 4, 32, 3>(p, b, width, height, o, out_rgb, out_T, n_contrib, st);
  if (gw == 4 && gh == 2) return launch_cfg<4, 2, 4, 32, 3>(p, b, width, height, o, out_rgb, out_T, n_contrib, st);
  if (gw == 2 && gh == 4) return launch_cfg<2, 4, 4, 32, 3>(p, b, width, height, o, out_rgb, out_T, n_contrib, st);
  if (gw == 4 && gh == 4) return launch_cfg<4, 4, 4, 32, 3>(p, b, width, height, o, out_rgb, out_T, n_contrib, st);
  set_error("tensor-core path supports groups 1x1, 2x2, 4x2, 2x4, 4x4 (got %dx%d)", gw, gh);
  return TGS_ERR_INVALID_ARGUMENT;
}

}  // namespace tgs
