// Bin and sort (Section 2 "Gaussian sorting"; Section 4.4.2 "Constructing the grouped Gaussian
// list"; Algorithm 1: one entry per (Gaussian, overlapped tile group) with a tile-membership mask,
// sorted by (group ID, depth)).
//
// The result equals an ascending LSD radix sort of the 64-bit keys (gid << 32) | bits(depth) with
// ties by Gaussian index. Every duplicate of a Gaussian carries the same depth, so the 32 depth
// bits are sorted once per visible Gaussian (4 stable 8-bit passes over n items) before the
// duplication; the duplicates are then emitted in that depth order and stably sorted by group id
// alone (ceil(log2 G / 8) passes over E items). A stable LSD sort is exactly this composition.
//
// Tile membership (beyond the paper; Section 6 cites tighter splat footprints as related work):
// a tile of a Gaussian's AABB tile range is a member only if the Gaussian's ellipse at the level
// where o e^power could reach 1/255 (widened for safety) meets the tile's pixel-centre box; an
// entry is emitted for a group only if one of its tiles is a member, and its mask holds the
// member tiles. A dropped (Gaussian, tile) pair fails the pruning test at every pixel of the
// tile, so the image does not change; the lists, the sort and the rasterizer's gathers shrink.
// Per tile row the member tiles are one run (the ellipse is convex), found from the ellipse's
// x-extent in the row's band; the test is a decision about which entries exist, taken in FP32
// with every operation rounded on its own in a fixed order, so that it is reproducible bit for bit.
//
// Stages (sizes read from device memory, so no host round trip is needed):
//   depth keys of the visible Gaussians + their digit histograms -> 4 radix passes (depth order)
//   -> per Gaussian, its number of entries (O(tile rows) of arithmetic) -> exclusive prefix of the
//   counts (total = entries the frame needs) -> emit (group id, index, mask) in depth order, with
//   the histograms of the group-id digits -> radix passes over the group-id digits carrying index
//   and mask -> group ranges from the sorted group ids (and the optional 64-bit keys).
// Every radix pass and the prefix are single kernels: a tile's offsets come from the earlier tiles
// by decoupled look-back (bounded waits) instead of separate histogram and scan kernels.
#include <algorithm>
#include <atomic>

#include "tgs_internal.cuh"

namespace tgs {
namespace {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;  // 8 warps
constexpr int kSortItems = 16;     // per thread
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 items per tile
constexpr int kMaxPasses = 4;
// threads and items per thread of the radix passes (tiles of threads x items)
constexpr int kDepthThreads = 256;
constexpr int kDepthItems = 16;
constexpr int kGidThreads = 256;
constexpr int kGidItems = 16;
// Look-back status words: 2 flag bits over a 30-bit count (sizes are limited to < 2^30).
constexpr uint32_t kFlagAgg = 1u << 30;     // the tile's own count is published
constexpr uint32_t kFlagPrefix = 2u << 30;  // the inclusive prefix up to the tile is published
constexpr uint32_t kValMask = (1u << 30) - 1u;
constexpr uint64_t kFlagAgg64 = 1ull << 62, kFlagPrefix64 = 2ull << 62;
constexpr uint64_t kValMask64 = (1ull << 62) - 1ull;

// The bounded waits of one bin sort call: where a wait that runs out is reported (the device error
// word, sticky until read, and the call's own failure word in its workspace, cleared at the start of
// every call), and the limit of one wait.
struct WaitCtl {
  int32_t* err;
  int32_t* failed;
  uint64_t limit_ns;
};

__device__ __forceinline__ void wait_expired(const WaitCtl& wc) {
  if (wc.err) atomicExch(wc.err, TGS_ERR_TIMEOUT);
  atomicExch(wc.failed, 1);
}

__device__ __forceinline__ int64_t live_count(const int64_t* count_dev, int64_t count_host,
                                              int64_t cap) {
  if (!count_dev) return count_host;
  const int64_t c = *count_dev;
  return (c < 0 || c > cap) ? 0 : c;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive scan over the block's THREADS threads (all of them call it); `tmp` holds THREADS / 32
// values.
template <typename T, int THREADS = kSortThreads>
__device__ __forceinline__ T block_excl_scan(T v, T* tmp, T* total = nullptr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T incl = warp_incl_scan(v);
  __syncthreads();
  if (lane == 31) tmp[warp] = incl;
  __syncthreads();
  T add = 0, all = 0;
#pragma unroll
  for (int w = 0; w < THREADS / 32; ++w) {
    const T t = tmp[w];
    if (w < warp) add += t;
    all += t;
  }
  if (total) *total = all;
  return incl - v + add;
}

// Decoupled look-back (a single-pass scan over tiles taken in launch order): publishes this tile's
// count for slot `d`, then adds the counts of the earlier tiles until one with a published
// inclusive prefix. The status words of up to kWindow earlier tiles are read at once (one memory
// round trip per window). Tiles are numbered by an atomic ticket taken when the block starts, so
// every earlier tile belongs to a block that is already running. A wait longer than the limit
// records TGS_ERR_TIMEOUT, marks the call failed and stops; the tile then publishes a prefix that is
// short (never long), so every position derived from it stays below the true one, and the kernels
// that follow turn the failed call into empty bins.
constexpr int kWindow = 16;

__device__ uint32_t lookback32(uint32_t* status, int tile, int slots, int d, uint32_t mine,
                               const WaitCtl& wc) {
  volatile uint32_t* st = status;
  if (tile == 0) {
    st[d] = kFlagPrefix | mine;
    return 0u;
  }
  st[(size_t)tile * slots + d] = kFlagAgg | mine;
  uint32_t excl = 0;
  uint64_t t0 = 0;
  int t = tile - 1;
  for (;;) {
    uint32_t w[kWindow];
#pragma unroll
    for (int k = 0; k < kWindow; ++k)
      w[k] = (t - k >= 0) ? (uint32_t)st[(size_t)(t - k) * slots + d] : +kFlagPrefix;  // before tile 0: 0
    int k = 0;
    bool done = false;
#pragma unroll
    for (int kk = 0; kk < kWindow; ++kk) {
      if (done || k != kk) continue;
      const uint32_t f = w[kk] & ~kValMask;
      if (f == 0u) continue;  // not published yet: poll again from here
      excl += w[kk] & kValMask;
      if (f == kFlagPrefix) done = true;
      else ++k;
    }
    if (done) break;
    t -= k;
    if (k == 0) {  // no progress in this round
      const uint64_t now = globaltimer_ns();
      if (t0 == 0) t0 = now;
      if (now - t0 > wc.limit_ns) {
        wait_expired(wc);
        break;
      }
    }
  }
  st[(size_t)tile * slots + d] = kFlagPrefix | (excl + mine);
  return excl;
}

// The same for one 64-bit value per tile, done by one warp: lane k reads tile t - k.
__device__ uint64_t lookback64_warp(uint64_t* status, int tile, uint64_t mine, const WaitCtl& wc) {
  volatile uint64_t* st = status;
  const int lane = threadIdx.x & 31;
  if (tile == 0) {
    if (lane == 0) st[0] = kFlagPrefix64 | mine;
    return 0ull;
  }
  if (lane == 0) st[tile] = kFlagAgg64 | mine;
  uint64_t excl = 0;
  uint64_t t0 = 0;
  int t = tile - 1;
  for (;;) {
    const uint64_t w = (t - lane >= 0) ? (uint64_t)st[t - lane] : +kFlagPrefix64;  // before tile 0: 0
    const uint64_t f = w & ~kValMask64;
    const uint32_t not_ready = __ballot_sync(0xffffffffu, f == 0ull);
    const uint32_t prefix = __ballot_sync(0xffffffffu, f == kFlagPrefix64);
    // lanes usable in order: up to the first prefix, stopping at the first unpublished one
    const uint32_t stop_nr = not_ready ? (__ffs(not_ready) - 1) : 32u;
    const uint32_t stop_pf = prefix ? (__ffs(prefix) - 1) : 32u;
    const bool done = stop_pf < stop_nr;
    const uint32_t used = done ? stop_pf + 1 : stop_nr;  // lanes 0 .. used-1 are added
    uint64_t v = (lane < (int)used) ? (w & kValMask64) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    excl += v;
    if (done) break;
    t -= (int)used;
    if (used == 0) {
      const uint64_t now = __shfl_sync(0xffffffffu, globaltimer_ns(), 0);
      if (t0 == 0) t0 = now;
      if (now - t0 > wc.limit_ns) {
        if (lane == 0) wait_expired(wc);
        break;
      }
    }
  }
  if (lane == 0) st[tile] = kFlagPrefix64 | (excl + mine);
  return excl;
}

// ---------------------------------------------------------------------------------------------
// Tile membership. With Q(d) = a dx^2 + 2 b dx dy + c dy^2 (the conic), a pair can matter only where
// o e^(-Q/2) >= 1/255. The test uses the level R = 2 (ln 255 + L(o) + kMemberMargin) with L(o) >=
// ln(o) read off the float's exponent and mantissa (k ln 2 + ln 2 / 2 if the mantissa is below
// sqrt 2, else (k + 1) ln 2) and widens every tile's pixel-centre box by kMemberEps px. In the band
// of tile row ty the ellipse Q <= R spans x in [xmin, xmax], attained at the band's points nearest
// to the ellipse's leftmost and rightmost points (dy = +-(b/c) Xmax, Xmax = sqrt(R c / det)); the
// member tiles of the row are the run whose widened boxes meet that span. Every operation is a
// single IEEE-rounded FP32 operation in a fixed order (the _rn intrinsics; one FMA pair for Kahan's
// determinant), so the result is reproducible bit for bit.
constexpr float kMemberEps = 0.0625f;
constexpr float kMemberMargin = 0.05f;

struct Member {
  float mx, my, ia, b, det, aR, Xmax, Ymax, bc;
  bool all;   // degenerate conic: every tile of the range is a member
  bool none;  // o < 1/255: no tile is
};

__device__ __forceinline__ float clamp_rn(float v, float lo, float hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

__device__ __forceinline__ Member member_setup(float2 mu, float4 co) {
  Member g;
  g.mx = mu.x;
  g.my = mu.y;
  g.b = co.y;
  g.all = false;
  g.none = false;
  g.ia = g.det = g.aR = g.Xmax = g.Ymax = g.bc = 0.f;
  const float w = __fmul_rn(co.y, co.y);
  const float e = __fmaf_rn(-co.y, co.y, w);
  const float det = __fadd_rn(__fmaf_rn(co.x, co.z, -w), e);
  if (!(co.x > 0.f) || !(co.z > 0.f) || !(det > 0.f)) {
    g.all = true;
    return g;
  }
  const uint32_t bits = __float_as_uint(co.w);
  const int ex = (int)((bits >> 23) & 0xFFu);
  const uint32_t man = bits & 0x7FFFFFu;
  // L(o) = halves * (ln 2) / 2; 0x3504F3 is the mantissa of the largest float below sqrt 2
  const int halves = ex == 0 ? -250 : 2 * (ex - 127) + (man <= 0x3504F3u ? 1 : 2);
  const float L = __fmul_rn((float)halves, 0.3465736f);
  float t = __fadd_rn(5.5412636f, L);  // ln 255
  t = __fadd_rn(t, kMemberMargin);
  const float R = __fmul_rn(2.0f, t);
  if (!(R > 0.f)) {
    g.none = true;
    return g;
  }
  const float aR = __fmul_rn(co.x, R);
  const float cR = __fmul_rn(co.z, R);
  g.aR = aR;
  g.det = det;
  g.Ymax = __fsqrt_rn(__fdiv_rn(aR, det));
  g.Xmax = __fsqrt_rn(__fdiv_rn(cR, det));
  g.bc = __fdiv_rn(co.y, co.z);
  g.ia = __fdiv_rn(1.0f, co.x);
  return g;
}

// Member tiles [lo, hi] of tile row ty (lo > hi: none), before clipping to the tile range.
__device__ __forceinline__ int2 member_row(const Member& g, int ty) {
  const float y0 = __fsub_rn((float)(16 * ty), kMemberEps);
  const float y1 = __fadd_rn((float)(16 * ty + 15), kMemberEps);
  const float dy0 = __fsub_rn(y0, g.my);
  const float dy1 = __fsub_rn(y1, g.my);
  const float nY = -g.Ymax;
  const float lb = dy0 > nY ? dy0 : nY;
  const float ub = dy1 < g.Ymax ? dy1 : g.Ymax;
  if (!(lb <= ub)) return make_int2(1, 0);
  const float sx = __fmul_rn(g.bc, g.Xmax);
  const float yh = clamp_rn(-sx, lb, ub);
  const float yl = clamp_rn(sx, lb, ub);
  const float qh = __fsub_rn(g.aR, __fmul_rn(__fmul_rn(g.det, yh), yh));
  const float ql = __fsub_rn(g.aR, __fmul_rn(__fmul_rn(g.det, yl), yl));
  const float sh = __fsqrt_rn(qh > 0.f ? qh : 0.f);
  const float sl = __fsqrt_rn(ql > 0.f ? ql : 0.f);
  const float xh = __fmul_rn(__fsub_rn(sh, __fmul_rn(g.b, yh)), g.ia);
  const float xl = __fmul_rn(__fsub_rn(-sl, __fmul_rn(g.b, yl)), g.ia);
  const float xmax = __fadd_rn(g.mx, xh);
  const float xmin = __fadd_rn(g.mx, xl);
  const float fh = clamp_rn(__fmul_rn(__fadd_rn(xmax, kMemberEps), 0.0625f), -1e6f, 1e6f);
  const float fl = clamp_rn(__fmul_rn(__fsub_rn(xmin, 15.0f + kMemberEps), 0.0625f), -1e6f, 1e6f);
  return make_int2((int)ceilf(fl), (int)floorf(fh));
}

// Member tiles of row ty clipped to the tile range r (lo > hi: none); `use` = membership on.
__device__ __forceinline__ int2 row_run(const Member& g, bool use, const int4& r, int ty) {
  int lo = r.x, hi = r.z - 1;
  if (use && !g.all) {
    if (g.none) return make_int2(1, 0);
    const int2 m = member_row(g, ty);
    lo = max(lo, m.x);
    hi = min(hi, m.y);
  }
  return make_int2(lo, hi);
}

// The member runs of the (up to TGS_MAX_GROUP) tile rows of group row gy, clipped to the tile
// range (lo > hi: none).
struct RowRuns {
  int lo[TGS_MAX_GROUP], hi[TGS_MAX_GROUP];
};

__device__ __forceinline__ RowRuns row_runs(const Member& g, bool use, const int4& r, int gy, int gh) {
  RowRuns q;
#pragma unroll
  for (int t = 0; t < TGS_MAX_GROUP; ++t) {
    const int ty = gy * gh + t;
    int2 run = make_int2(1, 0);
    if (t < gh && ty >= r.y && ty < r.w) run = row_run(g, use, r, ty);
    q.lo[t] = run.x;
    q.hi[t] = run.y;
  }
  return q;
}

__device__ __forceinline__ void cswap(int& s0, int& e0, int& s1, int& e1) {
  if (s1 < s0) {
    const int ts = s0, te = e0;
    s0 = s1; e0 = e1; s1 = ts; e1 = te;
  }
}

// Number of groups of the row holding a member tile: the length of the union of the tile rows'
// group-column runs [lo / gw, hi / gw] (sorted by a 4-input network, then swept).
__device__ __forceinline__ uint32_t row_group_count(const RowRuns& q, int gw) {
  int s[TGS_MAX_GROUP], e[TGS_MAX_GROUP];
#pragma unroll
  for (int t = 0; t < TGS_MAX_GROUP; ++t) {
    const bool ok = q.lo[t] <= q.hi[t];
    s[t] = ok ? q.lo[t] / gw : 0x7fffffff;
    e[t] = ok ? q.hi[t] / gw : -1;
  }
  static_assert(TGS_MAX_GROUP == 4, "sorting network for four runs");
  cswap(s[0], e[0], s[1], e[1]);
  cswap(s[2], e[2], s[3], e[3]);
  cswap(s[0], e[0], s[2], e[2]);
  cswap(s[1], e[1], s[3], e[3]);
  cswap(s[1], e[1], s[2], e[2]);
  uint32_t total = 0;
  int end = -1;
#pragma unroll
  for (int t = 0; t < TGS_MAX_GROUP; ++t) {
    if (e[t] < s[t]) continue;  // empty (sorted last)
    if (s[t] > end) {
      total += (uint32_t)(e[t] - s[t] + 1);
      end = e[t];
    } else if (e[t] > end) {
      total += (uint32_t)(e[t] - end);
      end = e[t];
    }
  }
  return total;
}

// Member-tile mask of group gx of the row, bit (ty - gy gh) gw + (tx - gx gw).
__device__ __forceinline__ uint32_t row_group_mask(const RowRuns& q, int gx, int gw) {
  uint32_t m = 0;
#pragma unroll
  for (int t = 0; t < TGS_MAX_GROUP; ++t) {
    const int lo = max(q.lo[t], gx * gw), hi = min(q.hi[t], gx * gw + gw - 1);
    for (int tx = lo; tx <= hi; ++tx) m |= 1u << (t * gw + (tx - gx * gw));
  }
  return m;
}

// The warp's view of one visible Gaussian (lane j holds Gaussian j of the warp's 32): its index,
// tile range, membership constants and number of group rows (0 if it has no entry).
struct WarpGauss {
  uint32_t i;
  int4 r;
  Member g;
  uint32_t rows;
};

__device__ __forceinline__ WarpGauss warp_gauss(int64_t s, int64_t n, const uint32_t* order,
                                                const int4* rect, const float2* mean2d,
                                                const float4* conic_opacity, int gh, bool use) {
  WarpGauss w{};
  w.i = 0;
  w.r = make_int4(0, 0, 0, 0);
  w.rows = 0;
  if (s < n) {
    w.i = order[s];
    w.r = rect[w.i];
    if (w.r.z > w.r.x && w.r.w > w.r.y) {
      if (use) w.g = member_setup(mean2d[w.i], conic_opacity[w.i]);
      if (!(use && w.g.none)) w.rows = (uint32_t)((w.r.w - 1) / gh - w.r.y / gh + 1);
    }
  }
  return w;
}

// Smallest lane whose inclusive prefix exceeds k.
__device__ __forceinline__ int find_src(uint32_t incl, uint32_t k) {
  int lo = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    const uint32_t v = __shfl_sync(0xffffffffu, incl, lo + step - 1);
    if (v <= k) lo += step;
  }
  return lo;
}

// Sum, over the lanes [lo_k - k0, hi_k - k0) of a round, of the values whose warp inclusive scan is
// S (hi_k > lo_k, both inside the round).
__device__ __forceinline__ uint32_t lanes_sum(uint32_t S, uint32_t lo_k, uint32_t hi_k, uint32_t k0) {
  const uint32_t hi_v = __shfl_sync(0xffffffffu, S, (int)(hi_k - 1 - k0));
  const uint32_t lo_v = __shfl_sync(0xffffffffu, S, (int)(lo_k > k0 ? lo_k - 1 - k0 : 0));
  return hi_v - (lo_k > k0 ? lo_v : 0u);
}

// ---------------------------------------------------------------------------------------------
// One stable LSD radix pass (8-bit digit at `shift`) of (u32 key, u32 value) pairs, single kernel.
// `ghist` holds the digit's counts over all items (from a histogram kernel run before the passes).
// Each tile of 256 * ITEMS items: each warp ranks its 32 * ITEMS consecutive items by digit
// (match_any); warps are ordered, so
// the tile's items get their stable rank in digit order. The tile's offset per digit is the
// global start of the digit plus the counts of that digit in the earlier tiles (look-back). Items
// are staged in shared memory in digit order and written so that each digit's run is contiguous
// and consecutive threads store consecutive words.
// With MASK, a 16-bit payload (the entry's tile mask) travels with each item as well. THREADS is a
// multiple of the 256 digits: the first 256 threads also do the per-digit work. Larger tiles mean
// fewer tiles, hence a shorter look-back chain when all tiles run in one wave. The staging buffers
// are dynamic shared memory (onesweep_smem_bytes).
template <int THREADS, int ITEMS, bool MASK>
constexpr size_t onesweep_smem_bytes() {
  return (size_t)THREADS * ITEMS * (8 + (MASK ? 2 : 0));
}

template <int THREADS, int ITEMS, bool MASK>
__global__ void __launch_bounds__(THREADS) k_onesweep(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
    const uint16_t* __restrict__ masks_in, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, uint16_t* __restrict__ masks_out, const int64_t* count_dev,
    int64_t count_host, int64_t cap, int shift, const uint32_t* __restrict__ ghist,
    uint32_t* __restrict__ status, int* __restrict__ tile_counter, WaitCtl wc) {
  static_assert(THREADS % kRadix == 0, "THREADS must be a multiple of the digit count");
  constexpr int W = THREADS / 32;
  constexpr int TILE = THREADS * ITEMS;
  __shared__ uint32_t wcount[W][kRadix];  // per warp and digit: count, then exclusive offset
  __shared__ uint32_t dstart[kRadix];     // tile-local start of each digit's run
  __shared__ uint32_t boff[kRadix];       // global start of this tile's run of each digit
  __shared__ uint32_t tmp[W];
  extern __shared__ __align__(16) uint8_t stage_raw[];
  uint32_t* skey = reinterpret_cast<uint32_t*>(stage_raw);
  uint32_t* sval = skey + TILE;
  uint16_t* smask = reinterpret_cast<uint16_t*>(sval + TILE);
  __shared__ int s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1);
  for (int k = threadIdx.x; k < W * kRadix; k += THREADS) (&wcount[0][0])[k] = 0;
  __syncthreads();
  const int tile = s_tile;
  const int64_t count = live_count(count_dev, count_host, cap);
  const int64_t block_base = (int64_t)tile * TILE;
  if (block_base >= count) return;  // uniform per block; later tickets are past the end too
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t key[ITEMS], val[ITEMS], rank[ITEMS];
  uint16_t msk[MASK ? ITEMS : 1];
  int dig[ITEMS];
  // all loads first, so that they are in flight together (the ranking below synchronizes the warp
  // between items)
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const int64_t i = block_base + (int64_t)warp * (32 * ITEMS) + r * 32 + lane;
    const bool valid = i < count;
    key[r] = valid ? keys_in[i] : 0u;
    val[r] = valid ? vals_in[i] : 0u;
    if (MASK) msk[MASK ? r : 0] = valid ? masks_in[i] : (uint16_t)0;
  }
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const int64_t i = block_base + (int64_t)warp * (32 * ITEMS) + r * 32 + lane;
    const bool valid = i < count;
    const int d = valid ? (int)((key[r] >> shift) & (kRadix - 1)) : kRadix;
    dig[r] = d;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = __popc(peers & lt_mask);
    uint32_t base = 0;
    if (valid) base = wcount[warp][d];
    __syncwarp();
    if (valid && before == 0) wcount[warp][d] = base + __popc(peers);
    __syncwarp();
    rank[r] = base + before;
  }
  __syncthreads();
  // per digit (the first 256 threads, one each): exclusive offsets over warps and the tile total
  const int d = threadIdx.x;
  const bool digit_thread = d < kRadix;
  uint32_t total = 0;
  if (digit_thread) {
#pragma unroll 8
    for (int w = 0; w < W; ++w) {
      const uint32_t c = wcount[w][d];
      wcount[w][d] = total;
      total += c;
    }
  }
  const uint32_t excl_tiles = digit_thread ? lookback32(status, tile, kRadix, d, total, wc) : 0u;
  const uint32_t gstart = block_excl_scan<uint32_t, THREADS>(digit_thread ? ghist[d] : 0u, tmp);
  const uint32_t ds = block_excl_scan<uint32_t, THREADS>(total, tmp);
  if (digit_thread) {
    dstart[d] = ds;
    boff[d] = gstart + excl_tiles;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const int dd = dig[r];
    if (dd < kRadix) {
      const uint32_t p = dstart[dd] + wcount[warp][dd] + rank[r];
      skey[p] = key[r];
      sval[p] = val[r];
      if (MASK) smask[p] = msk[MASK ? r : 0];
    }
  }
  __syncthreads();
  const int nvalid = (int)min((int64_t)TILE, count - block_base);
  for (int i = threadIdx.x; i < nvalid; i += THREADS) {
    const uint32_t k = skey[i];
    const int dd = (int)((k >> shift) & (kRadix - 1));
    const uint32_t pos = boff[dd] + (uint32_t)i - dstart[dd];
    if (pos >= (uint32_t)count) continue;  // only after an expired look-back (offsets then short)
    keys_out[pos] = k;
    vals_out[pos] = sval[i];
    if (MASK) masks_out[pos] = smask[i];
  }
}

// Launches one radix pass with the tiling of THREADS x ITEMS items per tile.
template <int THREADS, int ITEMS, bool MASK>
tgs_status launch_onesweep(int blocks, cudaStream_t st, const uint32_t* keys_in, const uint32_t* vals_in,
                           const uint16_t* masks_in, uint32_t* keys_out, uint32_t* vals_out,
                           uint16_t* masks_out, const int64_t* count_dev, int64_t cap, int shift,
                           const uint32_t* ghist, uint32_t* status, int* tile_counter,
                           const WaitCtl& wc) {
  constexpr size_t smem = onesweep_smem_bytes<THREADS, ITEMS, MASK>();
  auto* k = k_onesweep<THREADS, ITEMS, MASK>;
  // static + dynamic shared memory may exceed the default 48 KB: opt in to the dynamic part
  TGS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k<<<blocks, THREADS, smem, st>>>(keys_in, vals_in, masks_in, keys_out, vals_out, masks_out,
                                   count_dev, 0, cap, shift, ghist, status, tile_counter, wc);
  TGS_CHECK_LAUNCH("k_onesweep");
  return TGS_OK;
}

// ---------------------------------------------------------------------------------------------
// Binning kernels.

// Depth keys of the visible Gaussians, compacted in index order (a single-pass stable compaction:
// tile offsets by look-back), the visible count, and the histograms of the four 8-bit key digits.
// Each warp counts into its own shared histograms so shared atomics of different warps do not
// collide.
__global__ void __launch_bounds__(kSortThreads) k_depth_keys(
    int n, const int* __restrict__ radius, const float* __restrict__ depth,
    uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, int64_t* __restrict__ visible,
    uint32_t* __restrict__ ghist, uint64_t* __restrict__ status, int* __restrict__ tile_counter,
    WaitCtl wc) {
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t h[W][4 * kRadix];
  __shared__ uint32_t cnt[kSortItems][W];  // visible items per (round, warp), then their offsets
  __shared__ uint64_t s_prefix;
  __shared__ int s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1);
  for (int k = threadIdx.x; k < W * 4 * kRadix; k += kSortThreads) (&h[0][0])[k] = 0;
  __syncthreads();
  const int tile = s_tile;
  const int64_t base = (int64_t)tile * kSortTile;
  if (base >= n) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t* hw = h[warp];
  uint32_t key[kSortItems], ball[kSortItems];
  int rad[kSortItems];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {  // item r of thread t: base + r * 256 + t
    const int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
    rad[r] = i < n ? radius[i] : 0;
    // depth > near_z > 0, so the IEEE bits of a visible depth are monotone in the depth
    key[r] = i < n ? __float_as_uint(depth[i]) : 0u;
  }
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const bool vis = rad[r] > 0;
    if (vis) {  // the two low digits are spread: plain shared atomics
      atomicAdd(&hw[(key[r] & 0xffu)], 1u);
      atomicAdd(&hw[kRadix + ((key[r] >> 8) & 0xffu)], 1u);
    }
    // the two high digits take few values over a frame: one atomic per distinct digit of the warp
#pragma unroll
    for (int p = 2; p < 4; ++p) {
      const int d = vis ? (int)((key[r] >> (8 * p)) & 0xffu) : -1;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      if (vis && (__ffs(peers) - 1) == lane) atomicAdd(&hw[p * kRadix + d], __popc(peers));
    }
    ball[r] = __ballot_sync(0xffffffffu, vis);
    if (lane == 0) cnt[r][warp] = __popc(ball[r]);
  }
  __syncthreads();
  // exclusive offsets in (round, warp) order = index order
  if (threadIdx.x < 32) {
    uint32_t v[kSortItems * W / 32];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kSortItems * W / 32; ++k) {
      v[k] = (&cnt[0][0])[threadIdx.x * (kSortItems * W / 32) + k];
      sum += v[k];
    }
    const uint32_t incl = warp_incl_scan(sum);
    uint32_t run = incl - sum;
#pragma unroll
    for (int k = 0; k < kSortItems * W / 32; ++k) {
      (&cnt[0][0])[threadIdx.x * (kSortItems * W / 32) + k] = run;
      run += v[k];
    }
    const uint64_t tile_total = __shfl_sync(0xffffffffu, incl, 31);
    const uint64_t pre = lookback64_warp(status, tile, tile_total, wc);
    if (threadIdx.x == 0) s_prefix = pre;
    if (base + kSortTile >= n && threadIdx.x == 0) *visible = (int64_t)(pre + tile_total);
  }
  __syncthreads();
  const uint64_t prefix = s_prefix;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    if ((ball[r] >> lane) & 1u) {
      const uint64_t pos = prefix + cnt[r][warp] + __popc(ball[r] & lt_mask);
      keys[pos] = key[r];
      vals[pos] = (uint32_t)(base + (int64_t)r * kSortThreads + threadIdx.x);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 4 * kRadix; k += kSortThreads) {
    uint32_t v = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) v += h[w][k];
    if (v) atomicAdd(&ghist[k], v);
  }
}

// Per visible Gaussian in depth order, its number of entries: the groups of its tile range that
// hold a member tile. A warp takes 32 consecutive Gaussians (staged in shared memory) and spreads
// their group rows over its lanes (lane k of a round takes row k of the warp's rows, locating its
// Gaussian by a binary search over the prefix of row counts), so a large splat's rows are counted
// in parallel. GW, GH > 0 fix the grouping at compile time (0: the run-time gw, gh).
template <int GW, int GH>
__global__ void __launch_bounds__(256) k_count_entries(
    const int64_t* __restrict__ visible, const uint32_t* __restrict__ order,
    const int4* __restrict__ rect, const float2* __restrict__ mean2d,
    const float4* __restrict__ conic_opacity, int gw_rt, int gh_rt, int use,
    const int32_t* __restrict__ failed, uint32_t* __restrict__ counts) {
  const int gw = GW > 0 ? GW : gw_rt, gh = GH > 0 ? GH : gh_rt;
  __shared__ WarpGauss sg_all[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = *visible;
  if (s - lane >= n) return;  // warp-uniform
  if (*failed) {  // the depth order has holes: no entries
    if (s < n) counts[s] = 0u;
    return;
  }
  const WarpGauss w = warp_gauss(s, n, order, rect, mean2d, conic_opacity, gh, use != 0);
  sg_all[warp][lane] = w;
  __syncwarp();
  const uint32_t incl = warp_incl_scan(w.rows);
  const uint32_t excl = incl - w.rows;
  const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
  uint32_t carry = 0;  // lane j: entries of Gaussian j counted so far
  for (uint32_t k0 = 0; k0 < total; k0 += 32) {
    const uint32_t k = k0 + lane;
    const int src = find_src(incl, k);
    const uint32_t src_excl = __shfl_sync(0xffffffffu, excl, src);
    uint32_t c = 0;
    if (k < total) {
      const WarpGauss& sg = sg_all[warp][src];
      const int gy = sg.r.y / gh + (int)(k - src_excl);
      c = row_group_count(row_runs(sg.g, use != 0, sg.r, gy, gh), gw);
    }
    const uint32_t S = warp_incl_scan(c);
    const uint32_t lo_k = max(excl, k0), hi_k = min(incl, k0 + 32u);
    const bool mine = w.rows > 0 && lo_k < hi_k;
    const uint32_t sum = lanes_sum(S, mine ? lo_k : k0, mine ? hi_k : k0 + 1u, k0);
    if (mine) carry += sum;
  }
  if (s < n) counts[s] = carry;
}

// Exclusive prefix of the entry counts in depth order (single pass with look-back); the last tile
// writes the total, the number of entries the frame needs.
__global__ void __launch_bounds__(kSortThreads) k_entry_offsets(
    const int64_t* __restrict__ visible, const uint32_t* __restrict__ counts,
    uint32_t* __restrict__ offsets, int64_t* __restrict__ total, uint64_t* __restrict__ status,
    int* __restrict__ tile_counter, WaitCtl wc) {
  __shared__ uint64_t tmp[kSortThreads / 32];
  __shared__ uint64_t s_prefix;
  __shared__ int s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1);
  __syncthreads();
  const int tile = s_tile;
  const int64_t n = *visible;
  const int64_t base = (int64_t)tile * kSortTile + (int64_t)threadIdx.x * kSortItems;
  if (n == 0 && tile == 0 && threadIdx.x == 0) *total = 0;
  if ((int64_t)tile * kSortTile >= n) return;
  uint32_t c[kSortItems];
  uint64_t sum = 0;
  if (base + kSortItems <= n) {  // 16 consecutive counts: four 16-byte loads
    const uint4* p = reinterpret_cast<const uint4*>(counts + base);
#pragma unroll
    for (int k = 0; k < kSortItems / 4; ++k) {
      const uint4 v = p[k];
      c[4 * k] = v.x; c[4 * k + 1] = v.y; c[4 * k + 2] = v.z; c[4 * k + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) c[k] = base + k < n ? counts[base + k] : 0u;
  }
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) sum += c[k];
  uint64_t tile_total = 0;
  uint64_t run = block_excl_scan<uint64_t>(sum, tmp, &tile_total);
  if (threadIdx.x < 32) {
    const uint64_t pre = lookback64_warp(status, tile, tile_total, wc);
    if (threadIdx.x == 0) s_prefix = pre;
  }
  __syncthreads();
  run += s_prefix;
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    if (base + k < n) offsets[base + k] = (uint32_t)min(run, (uint64_t)0xFFFFFFFFu);
    run += c[k];
  }
  if (base < n && base + kSortItems >= n) *total = (int64_t)run;  // the thread holding item n-1
}

// Emits the entries of each visible Gaussian, in depth order: for every group of its tile range
// with a member tile, (group id, index, mask), the Gaussian's run starting at its offset. The warp
// spreads its 32 Gaussians' group rows over its lanes as k_count_entries does (same arithmetic, so
// the same counts); a lane writes its row's groups in order, at the row's position in the
// Gaussian's run. The block also counts the group-id digits of its entries for the radix passes.
template <int GW, int GH>
__global__ void __launch_bounds__(256) k_emit(
    const int64_t* __restrict__ visible, const uint32_t* __restrict__ order,
    const int4* __restrict__ rect, const float2* __restrict__ mean2d,
    const float4* __restrict__ conic_opacity, const uint32_t* __restrict__ offsets,
    const int64_t* __restrict__ total_entries, int64_t cap, int gw_rt, int gh_rt, int GX, int use,
    int passes, const int32_t* __restrict__ failed, uint32_t* __restrict__ gkeys,
    uint32_t* __restrict__ vals, uint16_t* __restrict__ masks, uint32_t* __restrict__ ghist) {
  const int gw = GW > 0 ? GW : gw_rt, gh = GH > 0 ? GH : gh_rt;
  __shared__ uint32_t h[kMaxPasses * kRadix];
  __shared__ WarpGauss sg_all[8][32];
  for (int k = threadIdx.x; k < passes * kRadix; k += blockDim.x) h[k] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = *visible;
  if (*total_entries <= cap && s - lane < n && !*failed) {  // warp-uniform
    const WarpGauss w = warp_gauss(s, n, order, rect, mean2d, conic_opacity, gh, use != 0);
    sg_all[warp][lane] = w;
    __syncwarp();
    const uint32_t base = s < n ? offsets[s] : 0u;
    const uint32_t incl = warp_incl_scan(w.rows);
    const uint32_t excl = incl - w.rows;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    uint32_t carry = 0;  // lane j: entries of Gaussian j written so far
    for (uint32_t k0 = 0; k0 < total; k0 += 32) {
      const uint32_t k = k0 + lane;
      const int src = find_src(incl, k);
      const WarpGauss& sg = sg_all[warp][src];
      const uint32_t src_excl = __shfl_sync(0xffffffffu, excl, src);
      const uint32_t src_base = __shfl_sync(0xffffffffu, base, src);
      const uint32_t src_carry = __shfl_sync(0xffffffffu, carry, src);
      RowRuns q;
      uint32_t c = 0;
      int gy = 0;
      if (k < total) {
        gy = sg.r.y / gh + (int)(k - src_excl);
        q = row_runs(sg.g, use != 0, sg.r, gy, gh);
        c = row_group_count(q, gw);
      }
      const uint32_t S = warp_incl_scan(c);
      // this row's position in its Gaussian's run: the Gaussian's earlier rounds, then its rows
      // on lower lanes of this round
      const uint32_t first = src_excl > k0 ? src_excl - k0 : 0u;
      const uint32_t before_first = __shfl_sync(0xffffffffu, S, first > 0 ? (int)first - 1 : 0);
      uint32_t pos = src_base + src_carry + (S - c) - (first > 0 ? before_first : 0u);
      if (c > 0) {
        int gmin = 0x7fffffff, gmax = -1;
#pragma unroll
        for (int t = 0; t < TGS_MAX_GROUP; ++t)
          if (q.lo[t] <= q.hi[t]) {
            gmin = min(gmin, q.lo[t] / gw);
            gmax = max(gmax, q.hi[t] / gw);
          }
        for (int gx = gmin; gx <= gmax; ++gx) {
          const uint32_t m = row_group_mask(q, gx, gw);
          if (!m) continue;
          if (pos < (uint32_t)cap) {  // always, unless an expired look-back left the offsets short
            const int gid = gy * GX + gx;
            gkeys[pos] = (uint32_t)gid;
            vals[pos] = sg.i;
            masks[pos] = (uint16_t)m;
            for (int p = 0; p < passes; ++p) atomicAdd(&h[p * kRadix + ((gid >> (8 * p)) & 0xff)], 1u);
          }
          ++pos;
        }
      }
      const uint32_t lo_k = max(excl, k0), hi_k = min(incl, k0 + 32u);
      const bool mine = w.rows > 0 && lo_k < hi_k;
      const uint32_t sum = lanes_sum(S, mine ? lo_k : k0, mine ? hi_k : k0 + 1u, k0);
      if (mine) carry += sum;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < passes * kRadix; k += blockDim.x)
    if (h[k]) atomicAdd(&ghist[k], h[k]);
}

// Group ranges from the sorted group ids ([start, end) at the first and past the last entry of
// each group; the others stay (0, 0)) and the optional 64-bit keys. A call whose look-back ran out
// ends here with empty bins: no ranges and an entry count of 0. A frame that needs more entries
// than the capacity sets the optional overflow word.
__global__ void k_ranges(int64_t* __restrict__ total, int64_t cap, const int32_t* __restrict__ failed,
                         const uint32_t* __restrict__ gkeys, const uint32_t* __restrict__ vals,
                         const float* __restrict__ depth, uint32_t* __restrict__ ranges,
                         uint64_t* __restrict__ keys64, int32_t* __restrict__ overflow) {
  if (*failed) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *total = 0;
    return;
  }
  const int64_t E = *total;
  if (E > cap) {
    if (overflow && blockIdx.x == 0 && threadIdx.x == 0) atomicExch(overflow, 1);
    return;
  }
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t g = gkeys[e];
    if (e == 0 || gkeys[e - 1] != g) ranges[2 * (size_t)g] = (uint32_t)e;
    if (e == E - 1 || gkeys[e + 1] != g) ranges[2 * (size_t)g + 1] = (uint32_t)(e + 1);
    if (keys64) keys64[e] = ((uint64_t)g << 32) | __float_as_uint(depth[vals[e]]);
  }
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Workspace: the ping-pong buffers, then one region that is cleared at the start of every call
// (digit histograms, look-back status words, tile tickets).
struct WsLayout {
  size_t dkA, dkB, dvA, dvB, counts, offs, gkA, gkB, gvB, gmB;
  size_t zero_begin, hist_d, hist_g, stat_d, stat_g, stat_o, stat_c, tickets, visible, failed,
      zero_end;
  int nb_c, nb_d, nb_g, nb_o;
  size_t total;
};

int group_bits(int64_t G) {
  int bits = 0;
  while ((int64_t(1) << bits) < G) ++bits;
  return bits;
}

WsLayout layout(int64_t n, int64_t cap, int GX, int GY) {
  const int64_t G = (int64_t)GX * GY;
  WsLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  L.nb_c = (int)std::max<int64_t>(1, div_up(n, kSortTile));
  L.nb_d = (int)std::max<int64_t>(1, div_up(n, kDepthThreads * kDepthItems));
  L.nb_g = (int)std::max<int64_t>(1, div_up(cap, kGidThreads * kGidItems));
  L.nb_o = L.nb_c;
  const int gpasses = std::max(1, div_up(group_bits(G), kRadixBits));
  L.dkA = take(4 * (size_t)n);
  L.dkB = take(4 * (size_t)n);
  L.dvA = take(4 * (size_t)n);
  L.dvB = take(4 * (size_t)n);
  L.counts = take(4 * (size_t)n);
  L.offs = take(4 * (size_t)n);
  L.gkA = take(4 * (size_t)cap);
  L.gkB = take(4 * (size_t)cap);
  L.gvB = take(4 * (size_t)cap);
  L.gmB = take(2 * (size_t)cap);
  L.zero_begin = off;
  L.hist_d = take(4 * 4 * kRadix);
  L.hist_g = take(4 * (size_t)kMaxPasses * kRadix);
  L.stat_d = take(4 * (size_t)4 * L.nb_d * kRadix);
  L.stat_g = take(4 * (size_t)gpasses * L.nb_g * kRadix);
  L.stat_o = take(8 * (size_t)L.nb_o);
  L.stat_c = take(8 * (size_t)L.nb_c);
  L.tickets = take(4 * (4 + kMaxPasses + 2));
  L.visible = take(8);
  L.failed = take(4);
  L.zero_end = off;
  L.total = off;
  return L;
}

}  // namespace

size_t bin_sort_workspace_bytes(int64_t n, int64_t capacity, int GX, int GY) {
  return layout(n, capacity, GX, GY).total;
}

int32_t* bin_sort_failed_word(void* ws, int64_t n, int64_t capacity, int GX, int GY) {
  return reinterpret_cast<int32_t*>(static_cast<char*>(ws) + layout(n, capacity, GX, GY).failed);
}

static std::atomic<int64_t> g_lookback_limit_ns{kDefaultLookbackLimitNs};

int64_t set_lookback_limit_ns(int64_t ns) {
  return g_lookback_limit_ns.exchange(ns > 0 ? ns : kDefaultLookbackLimitNs);
}

tgs_status launch_bin_sort(const tgs_projected& p, int64_t n64, int width, int height, int gw, int gh,
                           bool membership, void* ws, size_t ws_bytes, const tgs_bins& b,
                           cudaStream_t st, int32_t* err_word, int32_t* overflow_word) {
  (void)ws_bytes;
  const int n = (int)n64;
  const int TX = div_up(width, kTile), TY = div_up(height, kTile);
  const int GX = div_up(TX, gw), GY = div_up(TY, gh);
  const int64_t G = (int64_t)GX * GY;
  const int64_t cap = b.capacity;
  TGS_CUDA(cudaMemsetAsync(b.ranges, 0, sizeof(uint32_t) * 2 * (size_t)G, st));
  if (n == 0) {
    TGS_CUDA(cudaMemsetAsync(b.num_entries, 0, sizeof(int64_t), st));
    return TGS_OK;
  }
  if (((uintptr_t)p.rect & 15)) return set_error("rect must be 16-byte aligned"), TGS_ERR_INVALID_ARGUMENT;
  if (membership && (((uintptr_t)p.mean2d & 7) || ((uintptr_t)p.conic_opacity & 15) ||
                     !p.mean2d || !p.conic_opacity))
    return set_error("tile membership needs mean2d (8-byte aligned) and conic_opacity (16-byte "
                     "aligned)"),
           TGS_ERR_INVALID_ARGUMENT;
  const WsLayout L = layout(n64, cap, GX, GY);
  char* w = static_cast<char*>(ws);
  auto* dkA = reinterpret_cast<uint32_t*>(w + L.dkA);
  auto* dkB = reinterpret_cast<uint32_t*>(w + L.dkB);
  auto* dvA = reinterpret_cast<uint32_t*>(w + L.dvA);
  auto* dvB = reinterpret_cast<uint32_t*>(w + L.dvB);
  auto* counts = reinterpret_cast<uint32_t*>(w + L.counts);
  auto* offs = reinterpret_cast<uint32_t*>(w + L.offs);
  auto* gkA = reinterpret_cast<uint32_t*>(w + L.gkA);
  auto* gkB = reinterpret_cast<uint32_t*>(w + L.gkB);
  auto* gvB = reinterpret_cast<uint32_t*>(w + L.gvB);
  auto* gmB = reinterpret_cast<uint16_t*>(w + L.gmB);
  auto* hist_d = reinterpret_cast<uint32_t*>(w + L.hist_d);
  auto* hist_g = reinterpret_cast<uint32_t*>(w + L.hist_g);
  auto* stat_d = reinterpret_cast<uint32_t*>(w + L.stat_d);
  auto* stat_g = reinterpret_cast<uint32_t*>(w + L.stat_g);
  auto* stat_o = reinterpret_cast<uint64_t*>(w + L.stat_o);
  auto* tickets = reinterpret_cast<int*>(w + L.tickets);
  const int4* rect = reinterpret_cast<const int4*>(p.rect);
  const float2* m2 = reinterpret_cast<const float2*>(p.mean2d);
  const float4* co = reinterpret_cast<const float4*>(p.conic_opacity);
  auto* failed = reinterpret_cast<int32_t*>(w + L.failed);
  const WaitCtl wc{err_word ? err_word : device_error_word(), failed,
                   (uint64_t)g_lookback_limit_ns.load()};
  TGS_CUDA(cudaMemsetAsync(w + L.zero_begin, 0, L.zero_end - L.zero_begin, st));

  // 1. depth order of the visible Gaussians: compacted keys + digit histograms, then four
  //    single-kernel radix passes over the visible count
  auto* visible = reinterpret_cast<int64_t*>(w + L.visible);
  auto* stat_c = reinterpret_cast<uint64_t*>(w + L.stat_c);
  k_depth_keys<<<L.nb_c, kSortThreads, 0, st>>>(n, p.radius, p.depth, dkA, dvA, visible, hist_d,
                                                stat_c, tickets + 4 + kMaxPasses + 1, wc);
  TGS_CHECK_LAUNCH("k_depth_keys");
  for (int pass = 0; pass < 4; ++pass) {
    const bool odd = pass & 1;
    const tgs_status s = launch_onesweep<kDepthThreads, kDepthItems, false>(
        L.nb_d, st, odd ? dkB : dkA, odd ? dvB : dvA, nullptr, odd ? dkA : dkB, odd ? dvA : dvB,
        nullptr, visible, n, 8 * pass, hist_d + pass * kRadix,
        stat_d + (size_t)pass * L.nb_d * kRadix, tickets + pass, wc);
    if (s != TGS_OK) return s;
  }
  const uint32_t* order = dvA;  // after an even number of passes

  // 2. entries per Gaussian in depth order and their exclusive prefix (total = needed entries)
  // the visible count is not known on the host: one warp per 32 of all n Gaussians, the warps
  // past the visible ones return at once
  const int grp = gw * 10 + gh;
  auto count_kernel = grp == 11 ? k_count_entries<1, 1> : grp == 22 ? k_count_entries<2, 2>
                    : grp == 42 ? k_count_entries<4, 2> : grp == 24 ? k_count_entries<2, 4>
                    : grp == 44 ? k_count_entries<4, 4> : k_count_entries<0, 0>;
  count_kernel<<<div_up(n, 256), 256, 0, st>>>(visible, order, rect, m2, co, gw, gh,
                                               membership ? 1 : 0, failed, counts);
  TGS_CHECK_LAUNCH("k_count_entries");
  k_entry_offsets<<<L.nb_o, kSortThreads, 0, st>>>(visible, counts, offs, b.num_entries, stat_o,
                                                   tickets + 4 + kMaxPasses, wc);
  TGS_CHECK_LAUNCH("k_entry_offsets");
  if (cap == 0) return TGS_OK;

  // 3. emit (group id, index, mask) in depth order. The buffers are arranged so that the sorted
  //    indices and masks end in b.vals and b.masks after an odd or even number of radix passes.
  const int passes = div_up(group_bits(G), kRadixBits);
  uint32_t* ek = (passes & 1) ? gkB : gkA;
  uint32_t* ev = (passes & 1) ? gvB : b.vals;
  uint16_t* em = (passes & 1) ? gmB : b.masks;
  uint32_t* ok = (passes & 1) ? gkA : gkB;
  uint32_t* ov = (passes & 1) ? b.vals : gvB;
  uint16_t* om = (passes & 1) ? b.masks : gmB;
  auto emit_kernel = grp == 11 ? k_emit<1, 1> : grp == 22 ? k_emit<2, 2> : grp == 42 ? k_emit<4, 2>
                   : grp == 24 ? k_emit<2, 4> : grp == 44 ? k_emit<4, 4> : k_emit<0, 0>;
  emit_kernel<<<div_up(n, 256), 256, 0, st>>>(visible, order, rect, m2, co, offs, b.num_entries, cap,
                                               gw, gh, GX, membership ? 1 : 0, passes, failed, ek,
                                               ev, em, hist_g);
  TGS_CHECK_LAUNCH("k_emit");

  // 4. stable sort by group id, carrying index and mask
  const uint32_t* gk = ek;
  for (int pass = 0; pass < passes; ++pass) {
    const bool odd = pass & 1;
    const tgs_status s = launch_onesweep<kGidThreads, kGidItems, true>(
        L.nb_g, st, odd ? ok : ek, odd ? ov : ev, odd ? om : em, odd ? ek : ok, odd ? ev : ov,
        odd ? em : om, b.num_entries, cap, 8 * pass, hist_g + pass * kRadix,
        stat_g + (size_t)pass * L.nb_g * kRadix, tickets + 4 + pass, wc);
    if (s != TGS_OK) return s;
    gk = odd ? ek : ok;
  }

  // 5. group ranges and the optional 64-bit keys
  const int rng_blocks = std::max(1, std::min(div_up(cap, 256), 152 * 16));
  k_ranges<<<rng_blocks, 256, 0, st>>>(b.num_entries, cap, failed, gk, b.vals, p.depth, b.ranges,
                                       b.keys, overflow_word);
  TGS_CHECK_LAUNCH("k_ranges");
  return TGS_OK;
}

}  // namespace tgs
