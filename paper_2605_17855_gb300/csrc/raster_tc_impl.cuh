// Grouped tensor-core rasterizer (Section 4.2 "Tensorizing the power computation" and Section 4.4.2
// "Grouped rasterization"; Algorithm 1, the per-group CTA loop), written for sm_103a with tcgen05.
//
// One CTA per tile group. The group's depth-sorted list is read in chunks of NB = 32 entries and
// consumed as jobs of up to NB packed rows per tile:
//   * producer warps (several, on interleaved super-chunks of kSuper chunks): gather a chunk's
//     Gaussians (mean, conic, opacity, colour, mask). For every member tile, the entries whose mask
//     bit is set are appended to the tile's rows of the open job (Section 4.4.2: "select Gaussian
//     entries whose bit mask includes t"); a job spans chunks until a tile's NB rows would
//     overflow, so jobs stay dense after the tile skip below. For each packed entry the producer
//     writes the Gaussian's coefficient row of the power expansion about the
//     tile's centre (o_x, o_y) = (16 tx + 8, 16 ty + 8). With pixel offsets (x, y) = (px - o_x,
//     py - o_y) and (mx, my) = mu' - o:
//        log2(o) + log2(e) * power = q . [x^2, xy, y^2, x, y, 1]
//        q = log2(e) * (-a/2, -b, -c/2, a mx + b my, b mx + c my, -(a mx^2 + 2 b mx my + c my^2)/2)
//            + (0, 0, 0, 0, 0, log2 o)
//     This is the expansion of Eq. tensorgs_power_scalar about a common origin, which makes the
//     power a true matrix product (the Q Phi of Section 4.2.2 with the per-pixel terms separated
//     from the per-Gaussian ones). q is split into FP16 hi + lo and the K dimension holds
//     [hi(6), lo(6), 0, 0, 0, 0] against features [f(6), f(6), 0, 0, 0, 0]: the zero padding of
//     Section 4.2.3 (exact), with the padding slots used for the lo half. |x|, |y| <= 8, so every
//     feature is an exact FP16 integer. Rows whose FP16 error bound is too large take a scalar
//     FP32 path in the epilogue instead. A producer's gathers run one chunk ahead of its packing
//     and its index/mask loads two.
//     Unless disabled, a producer also leaves out of a tile's packed rows every entry whose exact
//     maximum exponent over the tile's 16x16 pixel centres is below log2(1/255) by a margin (the
//     minimum of the conic's quadratic form over a box, in closed form): such an entry fails the
//     pruning test at every pixel of the tile, so the image is unchanged; the tile's MMA rows,
//     exponent loads and tests for it are saved (a 3-sigma AABB overlaps many tiles the Gaussian
//     cannot reach at alpha >= 1/255).
//   * MMA thread: per tile, D[128 px x 32] = A_h[128 x 16] * B_t[32 x 16]^T with
//     tcgen05.mma.cta_group::1.kind::f16 (M = 128, N = 32, K = 16), FP32 accumulators in tensor
//     memory in NST stages (two, or one when two CTAs share an SM); completion signalled through
//     tcgen05.commit on mbarriers.
//   * epilogue warpgroups (one per tile of a round): each thread owns one TMEM lane = one pixel in
//     each of the tile's two 128-pixel M blocks, streams the tile's exponents out of tensor memory
//     8 columns at a time with the next load in flight (4 at a time, single-buffered, in the
//     one-stage configurations, whose register budget is 48 per thread) and runs
//     the front-to-back blend of Section 2 in FP32: skip if alpha < 1/255 (tested in the log2
//     domain before the exp), alpha = min(0.99, 2^D), stop when T' < 1e-4 without blending.
// Each chunk is loaded from global memory once per group and reused by all member tiles
// (the cross-tile reuse of Section 4.4.2); packing a tile's entries keeps their order, hence each
// tile's front-to-back order (Section 4.4.2, numerical equivalence with per-tile rasterization).
// Termination: before each job the MMA thread checks whether every epilogue warp has finished
// all its pixels (T < 1e-4 or end of list); if so it stops issuing, raises a stop flag for the
// producers and signals the epilogue the index of the last job.
// Every wait on an mbarrier is bounded (2 s); on expiry the CTA records TGS_ERR_TIMEOUT in the
// device error word, drains its MMAs, frees its tensor memory and exits.
#pragma once
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>

#include "tgs_internal.cuh"

namespace tgs {
namespace {

constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr float kL255 = -7.994353436858858f;            // log2(1/255)
constexpr float kLog2AlphaMax = -0.014499569695115089f;  // log2(0.99)
// Rows whose FP16 hi/lo error bound 2^-22 * sum_k |q_k| max|f_k| exceeds this (in log2 units)
// are evaluated by the scalar FP32 path.
constexpr float kMaxWeightedCoef = 4096.0f;
// A (Gaussian, tile) pair is skipped when the largest exponent over the tile's pixel box is below
// log2(1/255) by more than this (log2 units), far above the FP16 exponent error.
constexpr float kCullMargin = 0.01f;
constexpr int kLBO = 128;  // bytes between the two K core matrices of an 8-row group
constexpr int kSBO = 256;  // bytes between 8-row groups
constexpr int NB = 32;     // list entries per chunk = MMA N
// Chunks per super-chunk: the unit a producer packs into its own jobs (a job spans chunks until a
// tile's NB rows are full), so that jobs stay dense after the tile skip.
constexpr int kSuper = 2;
// Job slots per producer for groups of up to four tiles.
constexpr int kRingSmall = 2;

// Job counters of the producers' rings, kept in registers (p is warp-uniform).
template <int N>
__device__ __forceinline__ int ring_get(const int (&k)[N], int p) {
  int v = k[0];
#pragma unroll
  for (int i = 1; i < N; ++i)
    if (p == i) v = k[i];
  return v;
}
template <int N>
__device__ __forceinline__ void ring_inc(int (&k)[N], int p) {
#pragma unroll
  for (int i = 0; i < N; ++i) k[i] += (p == i) ? 1 : 0;
}

__device__ __forceinline__ float inf_f() { return __int_as_float(0x7f800000); }

template <int GW, int GH, int NWG, int NPROD, int NST = 2>
struct Cfg {
  static constexpr int kStages = NST;  // accumulator stages in tensor memory
  static constexpr int kTiles = GW * GH;
  static constexpr int kRounds = kTiles / NWG;
  static_assert(kTiles % NWG == 0, "tiles must split evenly over warpgroups");
  static constexpr int kEpiWarps = 4 * NWG;
  static constexpr int kProdWarp0 = kEpiWarps;
  static constexpr int kMmaWarp = kEpiWarps + NPROD;
  static constexpr int kThreads = 32 * (kMmaWarp + 1);
  // each producer has a ring of kRing job slots (deeper for small groups, whose slots are small)
  static constexpr int kRing = GW * GH <= 4 ? kRingSmall : 2;
  static constexpr int kSlots = kRing * NPROD;
  static constexpr int kStageCols = NWG * 2 * NB;
  static constexpr int kTmemCols = NST * kStageCols;
  static_assert(kTmemCols == 32 || kTmemCols == 64 || kTmemCols == 128 || kTmemCols == 256 ||
                    kTmemCols == 512,
                "TMEM allocation must be a power of two in [32, 512]");
};

template <int TILES, int KB>
struct __align__(16) Slot {
  uint8_t B[TILES][KB][NB * 32];  // per tile and K block of 16, packed rows; K-major canonical,
                                  // no swizzle: (row/8)*256 + (k/8)*128 + (row%8)*16
  float4 rgbc[TILES][NB];     // packed entry k of tile t: colour, min(log2 o, log2 0.99)
  uint32_t gidx[TILES][NB];   // Gaussian of packed entry k of tile t (read for scalar rows only)
  uint16_t rel[TILES][NB];    // list position of packed entry k of tile t, relative to `base`
  uint32_t cnt[TILES];        // packed entries of tile t
  uint32_t sbits[TILES];      // bit k: packed entry k of tile t uses the scalar path
  int32_t base;               // list position (from the group start) of the job's first chunk
  int32_t last;               // the job closes its super-chunk
};

template <int TILES, int SLOTS, int KB>
struct __align__(1024) Smem {
  uint8_t A[KB][2][4096];  // per K block, the two 128-pixel M blocks of the feature operand
  Slot<TILES, KB> slot[SLOTS];
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

__device__ __forceinline__ uint32_t pack_b2(float lo_elem, float hi_elem) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo_elem, hi_elem);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Round to BF16 and back.
__device__ __forceinline__ float bf16_round(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

// The error word may be host-mapped memory (a batched frame's status word), so it is set with a
// plain store: every writer stores the same value.
__device__ __forceinline__ void record_abort(int* abort_flag, int32_t* err) {
  *reinterpret_cast<volatile int*>(abort_flag) = 1;
  if (err) *reinterpret_cast<volatile int32_t*>(err) = TGS_ERR_TIMEOUT;
}

// Blend state of one pixel. `thr` is log2(1/255) while the pixel is live and +inf once it has
// terminated, so the pruning test alone also skips finished pixels.
struct PixState {
  float T, r, g, b, thr;
  int last;
};

// Smallest value of the quadratic form Q(d) = d^T conic d over the box of offsets
// d in [dx0, dx1] x [dy0, dy1] (the pixel centres of a tile relative to the Gaussian's mean). Q is
// convex: its minimum is 0 if the box holds d = 0, else it lies on an edge, where the 1D minimum is
// at the clamped stationary point. Evaluated through the Cholesky factor, Q = (l11 dx + l12 dy)^2 +
// (l22 dy)^2, so the result is a sum of squares.
__device__ __forceinline__ float box_min_quadratic(float a, float b, float c, float3 L, float dx0,
                                                   float dx1, float dy0, float dy1) {
  if (dx0 <= 0.f && dx1 >= 0.f && dy0 <= 0.f && dy1 >= 0.f) return 0.f;
  auto q = [&](float dx, float dy) {
    const float u = fmaf(L.x, dx, L.y * dy), v = L.z * dy;
    return fmaf(u, u, v * v);
  };
  const float ia = 1.f / a, ic = 1.f / c;
  float m = q(dx0, fminf(fmaxf(-b * dx0 * ic, dy0), dy1));
  m = fminf(m, q(dx1, fminf(fmaxf(-b * dx1 * ic, dy0), dy1)));
  m = fminf(m, q(fminf(fmaxf(-b * dy0 * ia, dx0), dx1), dy0));
  m = fminf(m, q(fminf(fmaxf(-b * dy1 * ia, dx0), dx1), dy1));
  return m;
}

// Cholesky factor (l11, l12, l22) of the conic [a b; b c], conic = L^T L with L = [l11 l12; 0 l22]:
// from the hardware reciprocal square root, the determinant by Kahan's scheme.
__device__ __forceinline__ float3 conic_cholesky(float4 co) {
  const float inv = rsqrtf(co.x);
  const float w2 = co.y * co.y;
  const float det = fmaf(co.x, co.z, -w2) + fmaf(-co.y, co.y, w2);
  const float dp = fmaxf(det, 0.f);
  return make_float3(co.x * inv, co.y * inv, dp > 0.f ? dp * rsqrtf(dp) * inv : 0.f);
}

// Scalar FP32 exponents of a packed entry whose FP16 coefficients would be too inaccurate: the
// Gaussian's mean and conic are read again and the power evaluated through the conic's factor.
__device__ __noinline__ float2 scalar_exponents(float px0, float py0, float px1, float py1,
                                                float2 mu, float4 co) {
  const float3 L = conic_cholesky(co);
  const float lo2 = lg2(co.w);
  const float e0 = fmaf(power_fp32(L, __fsub_rn(px0, mu.x), __fsub_rn(py0, mu.y)), kLog2e, lo2);
  const float e1 = fmaf(power_fp32(L, __fsub_rn(px1, mu.x), __fsub_rn(py1, mu.y)), kLog2e, lo2);
  return make_float2(e0, e1);
}

// One front-to-back step (Section 2) for one pixel, branch-free: the pruning test against the
// pixel's live threshold predicates the update. D = log2(o e^power) already contains the opacity,
// so alpha = min(0.99, 2^D) = 2^min(D, log2 0.99). NC: track the last blended list position.
template <bool COUNT, bool NC>
__device__ __forceinline__ void blend_step(float e, const float4& rc, PixState& s, int pos,
                                           unsigned long long& passing) {
  const bool p = e >= s.thr;                 // alpha >= 1/255 and the pixel is live
  if (COUNT) passing += p;
  const float a = ex2(fminf(e, kLog2AlphaMax));
  const float Tn = fmaf(-s.T, a, s.T);       // T (1 - alpha)
  const bool term = p && (Tn < kTMin);       // early termination: this entry is not blended
  if (p && !term) {
    const float w = a * s.T;
    s.r = fmaf(w, rc.x, s.r);
    s.g = fmaf(w, rc.y, s.g);
    s.b = fmaf(w, rc.z, s.b);
    s.T = Tn;
    if (NC) s.last = pos;
  }
  if (term) s.thr = inf_f();
}

// One packed entry (column jj of granule g) blended into the thread's two pixels.
template <int TILES, int KB, bool COUNT, bool NC>
__device__ __forceinline__ void blend_column(float e0, float e1, int j, int base,
                                             const Slot<TILES, KB>& sl, int t, PixState& s0,
                                             PixState& s1, unsigned long long& evaluated,
                                             unsigned long long& passing) {
  if (COUNT) evaluated += (s0.thr < inf_f()) + (s1.thr < inf_f());
  const float4 rc = sl.rgbc[t][j];
  const int pos = NC ? base + (int)sl.rel[t][j] + 1 : 0;
  blend_step<COUNT, NC>(e0, rc, s0, pos, passing);
  blend_step<COUNT, NC>(e1, rc, s1, pos, passing);
}

// Blends one granule of W columns (packed entries W g .. W g + W - 1 of tile t) into the thread's
// two pixels. d[0..W-1] are pixel 0's exponents, d[W..2W-1] pixel 1's. The steps are predicated,
// not branched per column, so the exponentials and tests of different columns and pixels overlap;
// a granule that is cut by the end of the tile's packed entries only runs its valid columns.
// SC = false leaves out the scalar FP32 rows (for jobs that have none).
template <int TILES, int KB, bool COUNT, bool NC, int W = 8, bool SC = true>
__device__ __forceinline__ void blend_granule(const uint32_t (&d)[2 * W], int g, int cnt, uint32_t sb,
                                              int base, const Slot<TILES, KB>& sl, int t, int tx,
                                              int ty, int quarter, int lane,
                                              const float2* __restrict__ mean2d,
                                              const float4* __restrict__ conic_opacity, PixState& s0,
                                              PixState& s1, unsigned long long& evaluated,
                                              unsigned long long& passing,
                                              unsigned long long& slots) {
  if (COUNT) slots += 2 * W;
  float e0[W], e1[W];
#pragma unroll
  for (int jj = 0; jj < W; ++jj) {
    e0[jj] = __uint_as_float(d[jj]);
    e1[jj] = __uint_as_float(d[W + jj]);
  }
  const uint32_t sbg = (sb >> (W * g)) & ((1u << W) - 1u);
  if (SC && sbg) {  // rare: rows whose FP16 coefficients would be too inaccurate
    int lx0, ly0, lx1, ly1;
    lane_pixel(0, quarter * 32 + lane, lx0, ly0);
    lane_pixel(1, quarter * 32 + lane, lx1, ly1);
    const float px0 = (float)(tx * kTile + lx0), py0 = (float)(ty * kTile + ly0);
    const float px1 = (float)(tx * kTile + lx1), py1 = (float)(ty * kTile + ly1);
#pragma unroll
    for (int jj = 0; jj < W; ++jj)
      if ((sbg >> jj) & 1u) {
        const uint32_t gi = sl.gidx[t][W * g + jj];
        const float2 es = scalar_exponents(px0, py0, px1, py1, mean2d[gi], conic_opacity[gi]);
        e0[jj] = es.x;
        e1[jj] = es.y;
      }
  }
  const int ncols = cnt - W * g;  // >= 1; warp-uniform
  if (ncols >= W) {
#pragma unroll
    for (int jj = 0; jj < W; ++jj)
      blend_column<TILES, KB, COUNT, NC>(e0[jj], e1[jj], W * g + jj, base, sl, t, s0, s1, evaluated,
                                         passing);
  } else {
#pragma unroll
    for (int jj = 0; jj < W - 1; ++jj)
      if (jj < ncols)
        blend_column<TILES, KB, COUNT, NC>(e0[jj], e1[jj], W * g + jj, base, sl, t, s0, s1, evaluated,
                                           passing);
  }
}

// ---- set-up helpers shared by the single-frame and the batched kernel ------------------------

// The constant feature operand A (exact integers in FP16 and BF16), written by the whole CTA.
template <int TILES, int SLOTS, int KB, bool BF>
__device__ __forceinline__ void write_feature_operand(Smem<TILES, SLOTS, KB>& S) {
  for (int m = threadIdx.x; m < 256; m += blockDim.x) {
    const int h = m >> 7, row = m & 127;
    int lx, ly;
    lane_pixel(h, row, lx, ly);
    const float x = (float)(lx - 8), y = (float)(ly - 8);
    const float f[6] = {x * x, x * y, y * y, x, y, 1.f};  // exact in FP16 and BF16 (|f| <= 64)
    auto pk = [&](float a, float b) { return BF ? pack_b2(a, b) : pack_h2(a, b); };
    uint4 c0, c1;
    // K block 0: [f, f, 0, 0, 0, 0] (against hi | lo, or hi | mid)
    c0.x = pk(f[0], f[1]); c0.y = pk(f[2], f[3]); c0.z = pk(f[4], f[5]);
    c0.w = pk(f[0], f[1]);
    c1.x = pk(f[2], f[3]); c1.y = pk(f[4], f[5]); c1.z = 0u; c1.w = 0u;
    uint8_t* rowp = &S.A[0][h][(row >> 3) * kSBO + (row & 7) * 16];
    *reinterpret_cast<uint4*>(rowp) = c0;
    *reinterpret_cast<uint4*>(rowp + kLBO) = c1;
    if (KB == 2) {  // K block 1 (BF16): [f, 0 ...] against lo
      c0.w = 0u;
      c1 = make_uint4(0u, 0u, 0u, 0u);
      uint8_t* rowq = &S.A[KB - 1][h][(row >> 3) * kSBO + (row & 7) * 16];
      *reinterpret_cast<uint4*>(rowq) = c0;
      *reinterpret_cast<uint4*>(rowq + kLBO) = c1;
    }
  }
}

// Barriers and per-group flags in their initial state (thread 0 only).
template <class C, int TILES, int SLOTS, int KB>
__device__ __forceinline__ void init_group_state(Smem<TILES, SLOTS, KB>& S) {
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

// The barriers invalidated, so that init_group_state may use their memory again (thread 0, after a
// CTA barrier that follows the drain of every tensor-core operation).
template <int TILES, int SLOTS, int KB>
__device__ __forceinline__ void inval_group_state(Smem<TILES, SLOTS, KB>& S) {
  for (int s = 0; s < SLOTS; ++s) {
    mbar_inval(&S.full[s]);
    mbar_inval(&S.empty[s]);
  }
  for (int s = 0; s < 2; ++s) {
    mbar_inval(&S.tfull[s]);
    mbar_inval(&S.tempty[s]);
  }
  mbar_inval(&S.drain);
}

// One tile group of one frame: producers, MMA thread and epilogue warpgroups (all warps of the CTA
// call it). Tensor memory is allocated, the feature operand written and the group state
// initialized by the caller.
template <int GW, int GH, int NWG, int NPROD, int NST, bool BF, bool COUNT, bool NC>
__device__ __forceinline__ void raster_group(
    Smem<GW * GH, Cfg<GW, GH, NWG, NPROD, NST>::kSlots, BF ? 2 : 1>& S, const uint32_t tmem,
    const int gid, const uint32_t* __restrict__ ranges, const uint32_t* __restrict__ vals,
    const uint16_t* __restrict__ masks, const float2* __restrict__ mean2d,
    const float4* __restrict__ conic_opacity, const float* __restrict__ rgb, int width, int height,
    int GX, float3 bg, float* __restrict__ out_rgb, float* __restrict__ out_T,
    int* __restrict__ n_contrib, unsigned long long* __restrict__ counters,
    int32_t* __restrict__ err, int cull) {
  using C = Cfg<GW, GH, NWG, NPROD, NST>;
  constexpr int TILES = C::kTiles;
  constexpr int KB = BF ? 2 : 1;  // K blocks of 16: FP16 hi|lo, or BF16 hi|mid then lo
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gx = gid % GX, gy = gid / GX;
  volatile int* abort_flag = &S.abort;
  volatile int* stop_flag = &S.stop;

  const uint32_t list_start = ranges[2 * gid], list_end = ranges[2 * gid + 1];
  const int nchunks = (int)((list_end - list_start + NB - 1) / NB);

  if (warp >= C::kProdWarp0 && warp < C::kMmaWarp) {
    // ---- producers: gather, pack per tile, coefficient rows -------------------------------------
    // The list is cut into chunks of NB entries and the chunks into super-chunks of kSuper;
    // producer p takes super-chunks p, p + NPROD, ... . It packs the surviving entries of its
    // consecutive chunks into a job in its own ring of two slots until a tile's NB rows would
    // overflow, then closes the job and opens the next; the last job of a super-chunk is flagged.
    // Consumers take the super-chunks in order, so each tile still sees its entries in list
    // order. Software pipeline: the gathers of the next chunk and the index/mask loads of the one
    // after it are in flight while a chunk is packed.
    const int p = warp - C::kProdWarp0;
    const uint32_t lt_mask = (1u << lane) - 1u;
    auto chunk_of = [&](int u) {  // the u-th chunk of this producer
      return (p + (u / kSuper) * NPROD) * kSuper + u % kSuper;
    };
    auto load_index = [&](int q, uint32_t& idx, uint32_t& msk, bool& valid) {
      const uint32_t e = list_start + (uint32_t)q * NB + lane;
      valid = q < nchunks && e < list_end;
      idx = valid ? vals[e] : 0u;
      msk = valid ? (uint32_t)masks[e] : 0u;
    };
    struct Gathered {
      float2 mu;
      float4 co;
    };
    auto gather = [&](uint32_t idx, bool valid, Gathered& g) {
      g.mu = valid ? mean2d[idx] : make_float2(0.f, 0.f);
      g.co = valid ? conic_opacity[idx] : make_float4(0.f, 0.f, 0.f, 1.f);
    };
    int k = 0;  // jobs opened in this producer's ring
    int s = 0;  // slot of the open job
    // waits for the next slot of the ring and starts a job at chunk q; false: stopped or timed out
    auto open_job = [&](int q) -> bool {
      s = C::kRing * p + k % C::kRing;
      const int w = mbar_wait_or_stop(&S.empty[s], ((k / C::kRing) & 1) ^ 1, stop_flag, abort_flag,
                                      kWaitLimitNs);
      const unsigned wmax = __reduce_max_sync(0xffffffffu, (unsigned)w);
      if (wmax != 0u) {
        if (wmax == 2u) record_abort(&S.abort, err);
        return false;
      }
      auto& sl = S.slot[s];
      if (lane < TILES) {
        sl.cnt[lane] = 0u;
        sl.sbits[lane] = 0u;
      }
      if (lane == 0) sl.base = q * NB;
      __syncwarp();
      return true;
    };
    auto close_job = [&](bool last) {
      if (lane == 0) S.slot[s].last = last ? 1 : 0;
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.full[s]);
      ++k;
    };
    uint32_t idx_a, msk_a, idx_b, msk_b;
    bool val_a, val_b;
    load_index(chunk_of(0), idx_a, msk_a, val_a);
    Gathered g_a;
    gather(idx_a, val_a, g_a);
    load_index(chunk_of(1), idx_b, msk_b, val_b);
    for (int u = 0;; ++u) {
      const int q = chunk_of(u);
      if (q >= nchunks) break;
      // the MMA thread stopped: every pixel of the group has finished
      if (__shfl_sync(0xffffffffu, *stop_flag, 0) != 0) break;
      Gathered g_b;
      gather(idx_b, val_b, g_b);  // chunk u + 1
      uint32_t idx_c, msk_c;
      bool val_c;
      load_index(chunk_of(u + 2), idx_c, msk_c, val_c);
      if (u % kSuper == 0 && !open_job(q)) break;
      const bool last = u % kSuper == kSuper - 1 || q + 1 >= nchunks;
      const float3 colr = val_a ? make_float3(rgb[3 * idx_a], rgb[3 * idx_a + 1], rgb[3 * idx_a + 2])
                                : make_float3(0.f, 0.f, 0.f);
      const bool valid = val_a;
      const uint32_t msk = msk_a;
      const float2 mu = g_a.mu;
      const float4 co = g_a.co;
      const float lo2 = lg2(co.w);
      // Cholesky factor of the conic (the tile skip and the linear/constant terms)
      const float3 Lc = valid ? conic_cholesky(co) : make_float3(0.f, 0.f, 0.f);
      const float4 rgbc = make_float4(colr.x, colr.y, colr.z, fminf(lo2, kLog2AlphaMax));
      // bit t of `act`: the entry is packed into tile t
      uint32_t act = 0u;
#pragma unroll
      for (int t = 0; t < TILES; ++t) {
        const int tx = gx * GW + (t % GW), ty = gy * GH + (t / GW);
        bool active = valid && ((msk >> t) & 1u);
        if (active && cull) {
          // skip the pair if no pixel of the tile can reach alpha >= 1/255 (exact bound)
          const float mx = mu.x - (float)(tx * kTile), my = mu.y - (float)(ty * kTile);
          const float qmin = box_min_quadratic(co.x, co.y, co.z, Lc, -mx, 15.f - mx, -my, 15.f - my);
          active = fmaf(-0.5f * kLog2e, qmin, lo2) >= kL255 - kCullMargin;
        }
        act |= (active ? 1u : 0u) << t;
      }
      // a tile whose rows would overflow closes the job; the chunk then starts a new one
      {
        bool over = false;
#pragma unroll
        for (int t = 0; t < TILES; ++t)
          over |= S.slot[s].cnt[t] + __popc(__ballot_sync(0xffffffffu, (act >> t) & 1u)) > (uint32_t)NB;
        if (over) {
          close_job(false);
          if (!open_job(q)) break;
        }
      }
      auto& sl = S.slot[s];
      const uint32_t rel = (uint32_t)(q * NB + lane - sl.base);
#pragma unroll
      for (int t = 0; t < TILES; ++t) {
        const bool active = (act >> t) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, active);
        if (bal == 0u) continue;
        const int tx = gx * GW + (t % GW), ty = gy * GH + (t / GW);
        // active entries are appended to the tile's rows in list order
        const uint32_t c0 = sl.cnt[t];
        const uint32_t pos = c0 + __popc(bal & lt_mask);
        bool scalar = false;
        if (active) {
          uint4 r0 = make_uint4(0u, 0u, 0u, 0u), r1 = make_uint4(0u, 0u, 0u, 0u);
          uint4 r2 = make_uint4(0u, 0u, 0u, 0u);  // BF16: K block 1 (lo)
          const float mx = mu.x - (float)(tx * kTile + 8), my = mu.y - (float)(ty * kTile + 8);
          // (u, v) = L m: the linear and constant terms are formed from it (conic m = L^T L m and
          // m^T conic m = u^2 + v^2), which avoids the cancellation of the expanded products when
          // the tile is far from the centre of a thin splat
          const float uu = fmaf(Lc.x, mx, Lc.y * my), vv = Lc.z * my;
          float qc[6];
          qc[0] = -0.5f * co.x * kLog2e;
          qc[1] = -co.y * kLog2e;
          qc[2] = -0.5f * co.z * kLog2e;
          qc[3] = Lc.x * uu * kLog2e;
          qc[4] = fmaf(Lc.y, uu, Lc.z * vv) * kLog2e;
          qc[5] = fmaf(-0.5f * kLog2e, fmaf(uu, uu, vv * vv), lo2);
          const float wsum = 64.f * (fabsf(qc[0]) + fabsf(qc[1]) + fabsf(qc[2])) +
                             8.f * (fabsf(qc[3]) + fabsf(qc[4])) + fabsf(qc[5]);
          scalar = !(wsum <= kMaxWeightedCoef);
          if (!scalar && !BF) {  // FP16: q = hi + lo, residual <= 2^-22 |q|
            const __half2 h01 = __floats2half2_rn(qc[0], qc[1]),
                          h23 = __floats2half2_rn(qc[2], qc[3]),
                          h45 = __floats2half2_rn(qc[4], qc[5]);
            const float2 f01 = __half22float2(h01), f23 = __half22float2(h23),
                         f45 = __half22float2(h45);
            r0.x = *reinterpret_cast<const uint32_t*>(&h01);
            r0.y = *reinterpret_cast<const uint32_t*>(&h23);
            r0.z = *reinterpret_cast<const uint32_t*>(&h45);
            r0.w = pack_h2(qc[0] - f01.x, qc[1] - f01.y);
            r1.x = pack_h2(qc[2] - f23.x, qc[3] - f23.y);
            r1.y = pack_h2(qc[4] - f45.x, qc[5] - f45.y);
          } else if (!scalar) {  // BF16: q = hi + mid + lo, residual <= 2^-27 |q|
            float hi[6], mid[6], lo[6];
#pragma unroll
            for (int kk = 0; kk < 6; ++kk) {
              hi[kk] = bf16_round(qc[kk]);
              mid[kk] = bf16_round(qc[kk] - hi[kk]);
              lo[kk] = qc[kk] - hi[kk] - mid[kk];
            }
            r0 = make_uint4(pack_b2(hi[0], hi[1]), pack_b2(hi[2], hi[3]), pack_b2(hi[4], hi[5]),
                            pack_b2(mid[0], mid[1]));
            r1 = make_uint4(pack_b2(mid[2], mid[3]), pack_b2(mid[4], mid[5]), 0u, 0u);
            r2 = make_uint4(pack_b2(lo[0], lo[1]), pack_b2(lo[2], lo[3]), pack_b2(lo[4], lo[5]), 0u);
          }
          uint8_t* rowp = &sl.B[t][0][(pos >> 3) * kSBO + (pos & 7) * 16];
          *reinterpret_cast<uint4*>(rowp) = r0;
          *reinterpret_cast<uint4*>(rowp + kLBO) = r1;
          if (KB == 2) {
            uint8_t* rowq = &sl.B[t][KB - 1][(pos >> 3) * kSBO + (pos & 7) * 16];
            *reinterpret_cast<uint4*>(rowq) = r2;
            *reinterpret_cast<uint4*>(rowq + kLBO) = make_uint4(0u, 0u, 0u, 0u);
          }
          sl.rgbc[t][pos] = rgbc;
          sl.rel[t][pos] = (uint16_t)rel;
          if (scalar) sl.gidx[t][pos] = idx_a;
        }
        const uint32_t sb = __reduce_or_sync(0xffffffffu, (active && scalar) ? (1u << pos) : 0u);
        if (lane == 0) {
          sl.cnt[t] = c0 + (uint32_t)__popc(bal);
          sl.sbits[t] |= sb;
        }
        __syncwarp();
      }
      if (last) close_job(true);
      // rotate the pipeline
      g_a = g_b;
      idx_a = idx_b;
      msk_a = msk_b;
      val_a = val_b;
      idx_b = idx_c;
      msk_b = msk_c;
      val_b = val_c;
    }
  } else if (warp == C::kMmaWarp) {
    // ---- MMA issuer ---------------------------------------------------------------------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(128, NB, BF);
      int job = 0;
      bool failed = false;
      // jobs in list order: super-chunk sc comes from producer sc % NPROD, whose jobs for it run
      // until the one flagged last
      int kc[NPROD];
#pragma unroll
      for (int i = 0; i < NPROD; ++i) kc[i] = 0;
      const int nsuper = (nchunks + kSuper - 1) / kSuper;
      int sc = 0;
      while (sc < nsuper && !failed) {
        // every epilogue warp has finished all its pixels: no more work for this group
        if (*reinterpret_cast<volatile int*>(&S.done_warps) >= C::kEpiWarps) break;
        const int pr = sc % NPROD, kk = ring_get(kc, pr);
        const int s = C::kRing * pr + kk % C::kRing;
        if (!mbar_wait_bounded(&S.full[s], (kk / C::kRing) & 1, abort_flag, kWaitLimitNs)) {
          failed = true;
          break;
        }
        auto& sl = S.slot[s];
        const int lastj = sl.last;
        for (int r = 0; r < C::kRounds; ++r, ++job) {
          const int st = job % NST;
          if (!mbar_wait_bounded(&S.tempty[st], ((job / NST) & 1) ^ 1, abort_flag, kWaitLimitNs)) {
            failed = true;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int g = 0; g < NWG; ++g) {
            const int t = g + NWG * r;
            if (sl.cnt[t] == 0u) continue;
            const uint32_t col = (uint32_t)(st * C::kStageCols + (2 * g) * NB);
#pragma unroll
            for (int kb = 0; kb < KB; ++kb) {
              const uint64_t bdesc = smem_desc(smem_addr(&sl.B[t][kb][0]), kLBO, kSBO);
              const uint32_t acc = kb > 0 ? 1u : 0u;
              mma_f16(tmem + col, smem_desc(smem_addr(&S.A[kb][0][0]), kLBO, kSBO), bdesc, idesc, acc);
              mma_f16(tmem + col + NB, smem_desc(smem_addr(&S.A[kb][1][0]), kLBO, kSBO), bdesc, idesc,
                      acc);
            }
          }
          mma_commit(&S.tfull[st]);
        }
        if (!failed) mma_commit(&S.empty[s]);
        ring_inc(kc, pr);
        if (lastj) ++sc;
      }
      *stop_flag = 1;
      if (failed) {
        record_abort(&S.abort, err);
      } else {
        // end signal: complete the next tfull phase with a plain arrive after publishing its index
        const int st = job % NST;
        if (mbar_wait_bounded(&S.tempty[st], ((job / NST) & 1) ^ 1, abort_flag, kWaitLimitNs)) {
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
        const bool inside = tx * kTile + lx < width && ty * kTile + ly < height;
        ps[r][h] = PixState{1.f, 0.f, 0.f, 0.f, inside ? kL255 : inf_f(), 0};
        all &= !inside;
      }
      wdone[r] = __all_sync(0xffffffffu, all);
    }
    bool counted_done = false;
    unsigned long long evaluated = 0, passing = 0, slots = 0;
    int job = 0;
    bool finished = false;
    // the MMA thread's job order (super-chunks in turn, each from its producer's ring)
    int kc[NPROD];
#pragma unroll
    for (int i = 0; i < NPROD; ++i) kc[i] = 0;
    int sc = 0;
    while (!finished) {
      const int pr = sc % NPROD, kk = ring_get(kc, pr);
      const int s = C::kRing * pr + kk % C::kRing;
      int lastj = 0;
#pragma unroll
      for (int r = 0; r < C::kRounds; ++r) {
        const int st = job % NST;
        bool ok = mbar_wait_bounded(&S.tfull[st], (job / NST) & 1, abort_flag, kWaitLimitNs);
        if (!__all_sync(0xffffffffu, ok)) { record_abort(&S.abort, err); finished = true; break; }
        if (__shfl_sync(0xffffffffu, *reinterpret_cast<volatile int*>(&S.end_job), 0) == job) {
          finished = true;
          break;
        }
        if (r == 0) {
          // the slot's producer writes (colours, packing) are complete: the MMA thread waited on
          // the same phase before issuing this job
          ok = mbar_wait_bounded(&S.full[s], (kk / C::kRing) & 1, abort_flag, kWaitLimitNs);
          if (!__all_sync(0xffffffffu, ok)) { record_abort(&S.abort, err); finished = true; break; }
          lastj = S.slot[s].last;
        }
        ++job;
        tc_fence_after();
        const auto& sl = S.slot[s];
        const int t = wg + NWG * r;
        const int cnt = (int)sl.cnt[t];
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) +
                               (uint32_t)(st * C::kStageCols + (2 * wg) * NB);
        if (cnt > 0 && !wdone[r]) {
          const uint32_t sb = sl.sbits[t];
          const int base = sl.base;
          const int tx = gx * GW + (t % GW), ty = gy * GH + (t / GW);
          const int ngr = (cnt + 7) >> 3;  // 8-column granules holding the packed entries
          if constexpr (NST == 1) {
            // one accumulator stage (two CTAs per SM): granules load one at a time, the other
            // CTA's warps hide the latency
            // granules of 4 columns (8 registers), so that the epilogue fits the 48-register cap
            const int ngr4 = (cnt + 3) >> 2;
            // the granule loop is instantiated twice: with the scalar FP32 rows (only for a job whose
            // packed rows include one, sb != 0) and without, so that the common loop carries no
            // register pressure for the rare scalar evaluation (measured 5% faster on c2)
            auto granules = [&](auto scalar_rows) {
              for (int g = 0; g < ngr4; ++g) {
                uint32_t ga[8];
                __syncwarp();
                tmem_ld4x2_async(taddr + 4 * g, taddr + NB + 4 * g, ga);
                tmem_wait_ld8(ga);
                if (g + 1 == ngr4) {
                  tc_fence_before();
                  __syncwarp();
                  if (lane == 0) mbar_arrive(&S.tempty[st]);
                }
                blend_granule<TILES, KB, COUNT, NC, 4, decltype(scalar_rows)::value>(
                    ga, g, cnt, sb, base, sl, t, tx, ty, quarter, lane, mean2d, conic_opacity,
                    ps[r][0], ps[r][1], evaluated, passing, slots);
                // after every second granule: a warp whose 64 pixels have all finished releases the
                // stage and leaves the job (checking after every granule costs more than it saves)
                if ((g & 1) && g + 1 < ngr4 &&
                    __all_sync(0xffffffffu, ps[r][0].thr == inf_f() && ps[r][1].thr == inf_f())) {
                  tc_fence_before();
                  __syncwarp();
                  if (lane == 0) mbar_arrive(&S.tempty[st]);
                  break;
                }
              }
            };
            if (sb)
              granules(std::true_type{});
            else
              granules(std::false_type{});
          } else {
            // the same two instantiations as in the one-stage loop above
            auto granules8 = [&](auto scalar_rows) {
              uint32_t ga[16], gb[16];
              __syncwarp();
              tmem_ld8x2_async(taddr, taddr + NB, ga);
              tmem_wait_ld(ga);
              // granule g is blended while granule g + 1 is loading; the stage is released once its
              // last load has completed
              for (int g = 0; g < ngr; g += 2) {
                if (g + 1 < ngr) {
                  __syncwarp();
                  tmem_ld8x2_async(taddr + 8 * (g + 1), taddr + NB + 8 * (g + 1), gb);
                } else {
                  tc_fence_before();
                  __syncwarp();
                  if (lane == 0) mbar_arrive(&S.tempty[st]);
                }
                blend_granule<TILES, KB, COUNT, NC, 8, decltype(scalar_rows)::value>(
                    ga, g, cnt, sb, base, sl, t, tx, ty, quarter, lane, mean2d, conic_opacity,
                    ps[r][0], ps[r][1], evaluated, passing, slots);
                if (g + 1 < ngr) {
                  tmem_wait_ld(gb);
                  if (g + 2 < ngr) {
                    __syncwarp();
                    tmem_ld8x2_async(taddr + 8 * (g + 2), taddr + NB + 8 * (g + 2), ga);
                  } else {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&S.tempty[st]);
                  }
                  blend_granule<TILES, KB, COUNT, NC, 8, decltype(scalar_rows)::value>(
                      gb, g + 1, cnt, sb, base, sl, t, tx, ty, quarter, lane, mean2d,
                      conic_opacity, ps[r][0], ps[r][1], evaluated, passing, slots);
                  if (g + 2 < ngr) tmem_wait_ld(ga);
                }
              }
            };
            if (sb)
              granules8(std::true_type{});
            else
              granules8(std::false_type{});
          }
          wdone[r] = __all_sync(0xffffffffu, ps[r][0].thr == inf_f() && ps[r][1].thr == inf_f());
        } else {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&S.tempty[st]);
        }
        if (r == C::kRounds - 1) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&S.empty[s]);
          ring_inc(kc, pr);
          if (lastj) ++sc;
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
    for (int r = 0; r < C::kRounds; ++r) {
      const int t = wg + NWG * r;
      const int tx = gx * GW + (t % GW), ty = gy * GH + (t / GW);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int lx, ly;
        lane_pixel(h, quarter * 32 + lane, lx, ly);
        const int X = tx * kTile + lx, Y = ty * kTile + ly;
        if (X >= width || Y >= height) continue;
        const size_t p = (size_t)Y * width + X;
        const PixState& q = ps[r][h];
        out_rgb[p] = q.r + q.T * bg.x;
        out_rgb[HW + p] = q.g + q.T * bg.y;
        out_rgb[2 * HW + p] = q.b + q.T * bg.z;
        out_T[p] = q.T;
        if (n_contrib) n_contrib[p] = q.last;
      }
    }
    if (COUNT) {
      for (int o = 16; o > 0; o >>= 1) {
        evaluated += __shfl_xor_sync(0xffffffffu, evaluated, o);
        passing += __shfl_xor_sync(0xffffffffu, passing, o);
        slots += __shfl_xor_sync(0xffffffffu, slots, o);
      }
      if (lane == 0) {
        if (evaluated) atomicAdd(counters, evaluated);
        if (passing) atomicAdd(counters + 1, passing);
        if (slots) atomicAdd(counters + 2, slots);
      }
    }
  }

}

template <int GW, int GH, int NWG, int NPROD, int NST, bool BF, bool COUNT, bool NC>
__global__ void __launch_bounds__(Cfg<GW, GH, NWG, NPROD, NST>::kThreads, 2 / NST)
    k_raster_tc(const uint32_t* __restrict__ ranges, const uint32_t* __restrict__ vals,
                const uint16_t* __restrict__ masks, const float2* __restrict__ mean2d,
                const float4* __restrict__ conic_opacity, const float* __restrict__ rgb, int width,
                int height, int GX, float3 bg, float* __restrict__ out_rgb,
                float* __restrict__ out_T, int* __restrict__ n_contrib,
                unsigned long long* __restrict__ counters, int32_t* __restrict__ err, int cull) {
  using C = Cfg<GW, GH, NWG, NPROD, NST>;
  constexpr int TILES = C::kTiles;
  constexpr int SLOTS = C::kSlots;
  constexpr int KB = BF ? 2 : 1;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  auto& S = *reinterpret_cast<Smem<TILES, SLOTS, KB>*>(smem_raw);
  const int warp = threadIdx.x >> 5;
  // ---- set-up: feature operand A, barriers, tensor memory -------------------------------------
  write_feature_operand<TILES, SLOTS, KB, BF>(S);
  if (threadIdx.x == 0) init_group_state<C>(S);
  if (warp == C::kMmaWarp) {
    tmem_alloc(&S.tmem_base, C::kTmemCols);
    tmem_relinquish();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  raster_group<GW, GH, NWG, NPROD, NST, BF, COUNT, NC>(
      S, S.tmem_base, blockIdx.x, ranges, vals, masks, mean2d, conic_opacity, rgb, width, height, GX,
      bg, out_rgb, out_T, n_contrib, counters, err, cull);
  // ---- teardown -----------------------------------------------------------------------------
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == C::kMmaWarp) tmem_dealloc(S.tmem_base, C::kTmemCols);
}

// ---- batched rasterization: several frames in one persistent launch ---------------------------
// The work items are the (frame, tile group) pairs of all frames, numbered frame by frame. Each
// CTA takes the next item from a device counter until none is left, so frames of any size and
// resolution share the GPU in one launch; between items the CTA drains its tensor-core work and
// re-initializes its barriers. A bounded wait that expires inside an item is reported to the
// frame's status word (the launch's error word if it has none), and that CTA stops. Before an item
// of a frame is rendered, the frame's readiness flag (if any) must have reached its value: the CTA
// waits for it at most `wait_ns`; on expiry the frame's status word becomes TGS_ERR_TIMEOUT and its
// items are skipped (their pixels are not written), and items of a frame already marked failed are
// skipped at once. Once every item of a frame has been rendered or skipped, the CTA that finished
// its last item sets the frame's done word (if any) to its value, after a system-scope fence, so
// that a host thread polling it sees the frame's pixels and status final.
constexpr int kMaxBatchFrames = 32;

struct BatchFrame {
  const uint32_t* ranges;
  const uint32_t* vals;
  const uint16_t* masks;
  const float2* mean2d;
  const float4* conic_opacity;
  const float* rgb;
  float* out_rgb;
  float* out_T;
  const int32_t* ready;  // may be NULL
  int32_t* status;       // may be NULL (device or host-mapped memory)
  int32_t* done;         // may be NULL (device or host-mapped memory)
  int32_t ready_value, done_value;
  int32_t width, height, GX;
};

struct BatchArgs {
  BatchFrame f[kMaxBatchFrames];
  int32_t start[kMaxBatchFrames + 1];  // first work item of each frame; start[count] = total
  int32_t count;
};

// Waits until *flag >= value, at most limit_ns; true when it got there.
__device__ __forceinline__ bool wait_flag(const int32_t* flag, int32_t value, uint64_t limit_ns) {
  const volatile int32_t* f = flag;
  if (*f >= value) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    __nanosleep(2000);
    if (*f >= value) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

template <int GW, int GH, int NWG, int NPROD, int NST, bool BF>
__global__ void __launch_bounds__(Cfg<GW, GH, NWG, NPROD, NST>::kThreads, 2 / NST)
    k_raster_tc_batch(const __grid_constant__ BatchArgs B, int* __restrict__ next_item, float3 bg,
                      int32_t* __restrict__ err, int cull, uint64_t wait_ns) {
  // next_item[0]: the work counter; next_item[1 + f]: items of frame f finished
  using C = Cfg<GW, GH, NWG, NPROD, NST>;
  constexpr int TILES = C::kTiles;
  constexpr int SLOTS = C::kSlots;
  constexpr int KB = BF ? 2 : 1;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  auto& S = *reinterpret_cast<Smem<TILES, SLOTS, KB>*>(smem_raw);
  __shared__ int s_item, s_frame, s_run;
  const int warp = threadIdx.x >> 5;
  write_feature_operand<TILES, SLOTS, KB, BF>(S);
  if (threadIdx.x == 0) init_group_state<C>(S);
  if (warp == C::kMmaWarp) {
    tmem_alloc(&S.tmem_base, C::kTmemCols);
    tmem_relinquish();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const int total = B.start[B.count];
  while (true) {
    if (threadIdx.x == 0) {
      const int item = atomicAdd(next_item, 1);
      int f = 0;
      while (f + 1 < B.count && B.start[f + 1] <= item) ++f;
      int run = item < total ? 1 : 0;
      if (run) {
        const BatchFrame& fr = B.f[f];
        if (fr.status && *reinterpret_cast<volatile int32_t*>(fr.status) != TGS_OK) {
          run = 0;  // the frame has already failed
        } else if (fr.ready && !wait_flag(fr.ready, fr.ready_value, wait_ns)) {
          run = 0;
          if (fr.status) *reinterpret_cast<volatile int32_t*>(fr.status) = TGS_ERR_TIMEOUT;
        }
      }
      s_item = item;
      s_frame = f;
      s_run = run;
    }
    __syncthreads();
    const int item = s_item, f = s_frame;
    if (item >= total) break;
    if (s_run) {
      const BatchFrame& fr = B.f[f];
      raster_group<GW, GH, NWG, NPROD, NST, BF, false, false>(
          S, S.tmem_base, item - B.start[f], fr.ranges, fr.vals, fr.masks, fr.mean2d,
          fr.conic_opacity, fr.rgb, fr.width, fr.height, fr.GX, bg, fr.out_rgb, fr.out_T, nullptr,
          nullptr, fr.status ? fr.status : err, cull);
    }
    // every warp is done with the item and the MMA thread has drained its tensor-core work; the
    // item's pixels are visible device-wide before it is counted as finished
    __threadfence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0) {
      const BatchFrame& fr = B.f[f];
      const int items = B.start[f + 1] - B.start[f];
      if (fr.done && atomicAdd(next_item + 1 + f, 1) == items - 1) {
        __threadfence_system();
        *reinterpret_cast<volatile int32_t*>(fr.done) = fr.done_value;
      }
    }
    if (S.abort) break;  // a bounded wait expired: this CTA stops (uniform: read after the barrier)
    if (threadIdx.x == 0 && s_run) {
      inval_group_state(S);
      init_group_state<C>(S);
    }
    __syncthreads();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == C::kMmaWarp) tmem_dealloc(S.tmem_base, C::kTmemCols);
}

template <bool BF, int GW, int GH, int NWG, int NPROD, int NST = 2>
tgs_status launch_cfg(const tgs_projected& p, const tgs_bins& b, int width, int height,
                      const tgs_raster_opts& o, float* out_rgb, float* out_T, int32_t* n_contrib,
                      cudaStream_t st) {
  using Cf = Cfg<GW, GH, NWG, NPROD, NST>;
  using Sm = Smem<GW * GH, Cf::kSlots, BF ? 2 : 1>;
  static_assert(sizeof(Sm) + 1024 <= 227 * 1024, "shared memory of one CTA exceeds 227 KB");
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
  const int cull = (o.flags & TGS_RASTER_NO_CULL) ? 0 : 1;
  auto launch = [&](auto* k) -> tgs_status {
    TGS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<GX * GY, Cf::kThreads, smem, st>>>(b.ranges, b.vals, b.masks, m2, co, p.rgb, width, height,
                                           GX, bg, out_rgb, out_T, n_contrib, cnt, err, cull);
    return TGS_OK;
  };
  tgs_status s;
  if (count)
    s = n_contrib ? launch(k_raster_tc<GW, GH, NWG, NPROD, NST, BF, true, true>)
                  : launch(k_raster_tc<GW, GH, NWG, NPROD, NST, BF, true, false>);
  else
    s = n_contrib ? launch(k_raster_tc<GW, GH, NWG, NPROD, NST, BF, false, true>)
                  : launch(k_raster_tc<GW, GH, NWG, NPROD, NST, BF, false, false>);
  if (s != TGS_OK) return s;
  TGS_CHECK_LAUNCH("k_raster_tc");
  return TGS_OK;
}

// The launcher of one operand type (FP16 or BF16); each is instantiated in its own translation
// unit.
template <bool BF>
tgs_status launch_raster_tc_typed(const tgs_projected& p, const tgs_bins& b, int width, int height,
                                  int gw, int gh, const tgs_raster_opts& o, float* out_rgb,
                                  float* out_T, int32_t* n_contrib, cudaStream_t st) {
  if (((uintptr_t)p.mean2d & 7) || ((uintptr_t)p.conic_opacity & 15))
    return set_error("mean2d needs 8-byte and conic_opacity 16-byte alignment"), TGS_ERR_INVALID_ARGUMENT;
  // FP16 groups of up to 8 tiles and BF16 2x2 (about 83 KB of shared memory): one accumulator
  // stage of 256 tensor-memory columns and at most 48 registers, so that two CTAs share an SM and
  // hide each other's latency (measured faster than one CTA with two stages; BF16 2x2: 0.315 vs
  // 0.422 ms per 1.5M-Gaussian 1600x1064 frame). 1x1 (not limited by tensor memory), 4x4, and
  // BF16 4x2 / 2x4 (about 148 KB of shared memory: one CTA per SM) keep two stages
  constexpr int NST = BF ? 2 : 1;
  if (gw == 1 && gh == 1) return launch_cfg<BF, 1, 1, 1, 2>(p, b, width, height, o, out_rgb, out_T, n_contrib, st);
  if (gw == 2 && gh == 2) return launch_cfg<BF, 2, 2, 4, 3, 1>(p, b, width, height, o, out_rgb, out_T, n_contrib, st);
  if (gw == 4 && gh == 2) return launch_cfg<BF, 4, 2, 4, 3, NST>(p, b, width, height, o, out_rgb, out_T, n_contrib, st);
  if (gw == 2 && gh == 4) return launch_cfg<BF, 2, 4, 4, 3, NST>(p, b, width, height, o, out_rgb, out_T, n_contrib, st);
  // 4x4 BF16: two producers (four slots), so that the doubled coefficient tiles fit in shared memory
  if (gw == 4 && gh == 4)
    return launch_cfg<BF, 4, 4, 4, BF ? 2 : 3>(p, b, width, height, o, out_rgb, out_T, n_contrib, st);
  set_error("tensor-core path supports groups 1x1, 2x2, 4x2, 2x4, 4x4 (got %dx%d)", gw, gh);
  return TGS_ERR_INVALID_ARGUMENT;
}

template <bool BF, int GW, int GH, int NWG, int NPROD, int NST = 2>
tgs_status launch_batch_cfg(const RasterFrame* frames, int count, const tgs_raster_opts& o,
                            int* next_item, uint64_t wait_ns, cudaStream_t st, int share_div) {
  using Cf = Cfg<GW, GH, NWG, NPROD, NST>;
  using Sm = Smem<GW * GH, Cf::kSlots, BF ? 2 : 1>;
  BatchArgs B{};
  B.count = count;
  int64_t total = 0;
  for (int f = 0; f < count; ++f) {
    const RasterFrame& r = frames[f];
    const int TX = div_up(r.width, kTile), TY = div_up(r.height, kTile);
    const int GX = div_up(TX, GW), GY = div_up(TY, GH);
    if (((uintptr_t)r.p->mean2d & 7) || ((uintptr_t)r.p->conic_opacity & 15))
      return set_error("frame %d: mean2d needs 8-byte and conic_opacity 16-byte alignment", f),
             TGS_ERR_INVALID_ARGUMENT;
    BatchFrame& d = B.f[f];
    d.ranges = r.b->ranges;
    d.vals = r.b->vals;
    d.masks = r.b->masks;
    d.mean2d = reinterpret_cast<const float2*>(r.p->mean2d);
    d.conic_opacity = reinterpret_cast<const float4*>(r.p->conic_opacity);
    d.rgb = r.p->rgb;
    d.out_rgb = r.out_rgb;
    d.out_T = r.out_T;
    d.ready = r.ready;
    d.status = r.status;
    d.done = r.done;
    d.ready_value = r.ready_value;
    d.done_value = r.done_value;
    d.width = r.width;
    d.height = r.height;
    d.GX = GX;
    B.start[f] = (int32_t)total;
    total += (int64_t)GX * GY;
  }
  if (total >= (int64_t(1) << 31)) return set_error("batch has too many tile groups"), TGS_ERR_INVALID_ARGUMENT;
  B.start[count] = (int32_t)total;
  int dev = 0, smem_sm = 0, sms = 0;
  TGS_CUDA(cudaGetDevice(&dev));
  TGS_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  TGS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // residency as in the single-frame launch: co-resident CTAs never wait for tensor memory
  const int max_ctas = 512 / Cf::kTmemCols;
  size_t smem = sizeof(Sm) + 1024 + 64;
  smem = std::max(smem, (size_t)smem_sm / (max_ctas + 1) - 1024 + 16);
  auto* k = k_raster_tc_batch<GW, GH, NWG, NPROD, NST, BF>;
  TGS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // the residency the kernel is built for (its launch bounds and shared-memory floor): two CTAs
  // per SM with one accumulator stage. The occupancy query is not used: it assumes the default
  // L1 / shared-memory split, under which it reports one CTA per SM, while the driver picks the
  // split that fits two (as for the single-frame launch); a persistent grid of half the CTAs was
  // 1.4x slower.
  const int occ = 2 / NST;
  const int64_t slots = std::max<int64_t>(1, (int64_t)std::max(occ, 1) * sms / std::max(share_div, 1));
  const int grid = (int)std::min<int64_t>(std::max<int64_t>(total, 1), slots);
  TGS_CUDA(cudaMemsetAsync(next_item, 0, sizeof(int) * (1 + kMaxBatchFrames), st));
  const float3 bg = make_float3(o.bg[0], o.bg[1], o.bg[2]);
  const int cull = (o.flags & TGS_RASTER_NO_CULL) ? 0 : 1;
  k<<<grid, Cf::kThreads, smem, st>>>(B, next_item, bg, device_error_word(), cull, wait_ns);
  TGS_CHECK_LAUNCH("k_raster_tc_batch");
  return TGS_OK;
}

template <bool BF>
tgs_status launch_raster_tc_batch_typed(const RasterFrame* frames, int count, int gw, int gh,
                                        const tgs_raster_opts& o, int* next_item, uint64_t wait_ns,
                                        cudaStream_t st, int share_div) {
  constexpr int NST = BF ? 2 : 1;  // the configurations of the single-frame launch
  if (gw == 1 && gh == 1) return launch_batch_cfg<BF, 1, 1, 1, 2>(frames, count, o, next_item, wait_ns, st, share_div);
  if (gw == 2 && gh == 2) return launch_batch_cfg<BF, 2, 2, 4, 3, 1>(frames, count, o, next_item, wait_ns, st, share_div);
  if (gw == 4 && gh == 2) return launch_batch_cfg<BF, 4, 2, 4, 3, NST>(frames, count, o, next_item, wait_ns, st, share_div);
  if (gw == 2 && gh == 4) return launch_batch_cfg<BF, 2, 4, 4, 3, NST>(frames, count, o, next_item, wait_ns, st, share_div);
  if (gw == 4 && gh == 4)
    return launch_batch_cfg<BF, 4, 4, 4, BF ? 2 : 3>(frames, count, o, next_item, wait_ns, st, share_div);
  set_error("tensor-core path supports groups 1x1, 2x2, 4x2, 2x4, 4x4 (got %dx%d)", gw, gh);
  return TGS_ERR_INVALID_ARGUMENT;
}

}  // namespace
}  // namespace tgs
