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
// Stages (all kernels HBM-bound; sizes taken from device memory so no host round trip is needed):
//   depth keys + their digit histograms -> 4 radix passes -> exclusive prefix of the per-Gaussian
//   group counts (total = needed entries), with the per-group entry counts accumulated as a 2D
//   difference array -> group table (group ranges, histograms of the group-id digits) -> emit
//   (gid, index) in depth order -> radix passes over the group-id digits -> masks (from the tile
//   ranges) and the optional 64-bit keys.
// Every radix pass and the prefix are single kernels: a tile's offsets come from the earlier tiles
// by decoupled look-back (bounded waits) instead of separate histogram and scan kernels.
#include <algorithm>

#include "tgs_internal.cuh"

namespace tgs {
namespace {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;  // 8 warps
constexpr int kSortItems = 16;     // per thread
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 items per tile
constexpr int kMaxPasses = 4;
// items per thread of the radix passes (tiles of 256 x items)
constexpr int kDepthItems = 16;
constexpr int kGidItems = 16;
// Look-back status words: 2 flag bits over a 30-bit count (sizes are limited to < 2^30).
constexpr uint32_t kFlagAgg = 1u << 30;     // the tile's own count is published
constexpr uint32_t kFlagPrefix = 2u << 30;  // the inclusive prefix up to the tile is published
constexpr uint32_t kValMask = (1u << 30) - 1u;
constexpr uint64_t kFlagAgg64 = 1ull << 62, kFlagPrefix64 = 2ull << 62;
constexpr uint64_t kValMask64 = (1ull << 62) - 1ull;
constexpr uint64_t kLookbackLimitNs = 1000000000ull;  // 1 s

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

// Exclusive scan over the block's 256 threads (all of them call it); `tmp` holds 8 values.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* tmp, T* total = nullptr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T incl = warp_incl_scan(v);
  __syncthreads();
  if (lane == 31) tmp[warp] = incl;
  __syncthreads();
  T add = 0, all = 0;
#pragma unroll
  for (int w = 0; w < kSortThreads / 32; ++w) {
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
// records TGS_ERR_TIMEOUT and stops (the result is then wrong, but the kernel ends).
constexpr int kWindow = 16;

__device__ uint32_t lookback32(uint32_t* status, int tile, int slots, int d, uint32_t mine,
                               int32_t* err) {
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
      if (now - t0 > kLookbackLimitNs) {
        if (err) atomicExch(err, TGS_ERR_TIMEOUT);
        break;
      }
    }
  }
  st[(size_t)tile * slots + d] = kFlagPrefix | (excl + mine);
  return excl;
}

// The same for one 64-bit value per tile, done by one warp: lane k reads tile t - k.
__device__ uint64_t lookback64_warp(uint64_t* status, int tile, uint64_t mine, int32_t* err) {
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
      if (now - t0 > kLookbackLimitNs) {
        if (lane == 0 && err) atomicExch(err, TGS_ERR_TIMEOUT);
        break;
      }
    }
  }
  if (lane == 0) st[tile] = kFlagPrefix64 | (excl + mine);
  return excl;
}

// The per-entry outputs besides the Gaussian index: the mask of the group's member tiles inside the
// Gaussian's tile range and, optionally, the 64-bit key.
struct Finalize {
  const int4* rect;
  const float* depth;
  int gw, gh, GX;
  uint16_t* masks;
  uint64_t* keys64;  // may be NULL
};

__device__ __forceinline__ void entry_outputs(const Finalize& f, uint32_t pos, uint32_t g,
                                              uint32_t i) {
  const int4 r = f.rect[i];
  const int gx = (int)(g % (uint32_t)f.GX), gy = (int)(g / (uint32_t)f.GX);
  uint32_t m = 0;
  for (int ty = 0; ty < f.gh; ++ty)
    for (int tx = 0; tx < f.gw; ++tx) {
      const int X = gx * f.gw + tx, Y = gy * f.gh + ty;
      if (X >= r.x && X < r.z && Y >= r.y && Y < r.w) m |= 1u << (ty * f.gw + tx);
    }
  f.masks[pos] = (uint16_t)m;
  if (f.keys64) f.keys64[pos] = ((uint64_t)g << 32) | __float_as_uint(f.depth[i]);
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
template <int ITEMS>
__global__ void __launch_bounds__(kSortThreads) k_onesweep(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, const int64_t* count_dev,
    int64_t count_host, int64_t cap, int shift, const uint32_t* __restrict__ ghist,
    uint32_t* __restrict__ status, int* __restrict__ tile_counter, int32_t* __restrict__ err) {
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t wcount[W][kRadix];  // per warp and digit: count, then exclusive offset
  __shared__ uint32_t dstart[kRadix];     // tile-local start of each digit's run
  __shared__ uint32_t boff[kRadix];       // global start of this tile's run of each digit
  __shared__ uint32_t tmp[W];
  __shared__ uint32_t skey[kSortThreads * ITEMS], sval[kSortThreads * ITEMS];
  __shared__ int s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1);
  for (int k = threadIdx.x; k < W * kRadix; k += kSortThreads) (&wcount[0][0])[k] = 0;
  __syncthreads();
  const int tile = s_tile;
  const int64_t count = live_count(count_dev, count_host, cap);
  const int64_t block_base = (int64_t)tile * (kSortThreads * ITEMS);
  if (block_base >= count) return;  // uniform per block; later tickets are past the end too
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t key[ITEMS], val[ITEMS], rank[ITEMS];
  int dig[ITEMS];
  // all loads first, so that they are in flight together (the ranking below synchronizes the warp
  // between items)
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const int64_t i = block_base + (int64_t)warp * (32 * ITEMS) + r * 32 + lane;
    const bool valid = i < count;
    key[r] = valid ? keys_in[i] : 0u;
    val[r] = valid ? vals_in[i] : 0u;
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
  // per digit (one thread each): exclusive offsets over warps and the tile total
  static_assert(kSortThreads == kRadix, "one thread per digit");
  const int d = threadIdx.x;
  uint32_t total = 0;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const uint32_t c = wcount[w][d];
    wcount[w][d] = total;
    total += c;
  }
  const uint32_t excl_tiles = lookback32(status, tile, kRadix, d, total, err);
  const uint32_t gstart = block_excl_scan<uint32_t>(ghist[d], tmp);
  const uint32_t ds = block_excl_scan<uint32_t>(total, tmp);
  dstart[d] = ds;
  boff[d] = gstart + excl_tiles;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const int dd = dig[r];
    if (dd < kRadix) {
      const uint32_t p = dstart[dd] + wcount[warp][dd] + rank[r];
      skey[p] = key[r];
      sval[p] = val[r];
    }
  }
  __syncthreads();
  const int nvalid = (int)min((int64_t)(kSortThreads * ITEMS), count - block_base);
  for (int i = threadIdx.x; i < nvalid; i += kSortThreads) {
    const uint32_t k = skey[i];
    const int dd = (int)((k >> shift) & (kRadix - 1));
    const uint32_t pos = boff[dd] + (uint32_t)i - dstart[dd];
    keys_out[pos] = k;
    vals_out[pos] = sval[i];
  }
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
    int32_t* __restrict__ err) {
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
    const uint64_t pre = lookback64_warp(status, tile, tile_total, err);
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

// Exclusive prefix of the group counts of the Gaussians in depth order (single pass with
// look-back); the last tile writes the total, the number of entries the frame needs.
//
// It also counts the entries of every group: each Gaussian adds its rectangle of groups to a 2D
// difference array D over (GY + 1) x (GX + 1) cells (+1 at (gy0, gx0) and (gy1+1, gx1+1), -1 at
// (gy0, gx1+1) and (gy1+1, gx0)), whose 2D prefix sum is the per-group count. A tile accumulates
// D in shared memory and stores it to its own slice of `dslices` (no global atomics); if D does
// not fit (`dslices` == NULL) the tile adds into the global D (`dglobal`) instead.
__global__ void __launch_bounds__(kSortThreads) k_group_offsets(
    const int64_t* __restrict__ visible, const uint32_t* __restrict__ order,
    const int* __restrict__ radius,
    const int4* __restrict__ rect, int gw, int gh, int GXp1, int cells,
    uint64_t* __restrict__ offsets, int64_t* __restrict__ total, int32_t* __restrict__ dslices,
    int32_t* __restrict__ dglobal, uint64_t* __restrict__ status, int* __restrict__ tile_counter,
    int32_t* __restrict__ err) {
  extern __shared__ int32_t sD[];
  __shared__ uint64_t tmp[kSortThreads / 32];
  __shared__ uint64_t s_prefix;
  __shared__ int s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1);
  if (dslices)
    for (int k = threadIdx.x; k < cells; k += kSortThreads) sD[k] = 0;
  __syncthreads();
  const int tile = s_tile;
  const int64_t n = *visible;
  const int64_t base = (int64_t)tile * kSortTile + (int64_t)threadIdx.x * kSortItems;
  if (n == 0 && tile == 0 && threadIdx.x == 0) *total = 0;
  if ((int64_t)tile * kSortTile >= n) return;
  int32_t* D = dslices ? sD : dglobal;
  uint32_t c[kSortItems];
  int4 rc[kSortItems];
  uint64_t sum = 0;
  // loads first (the Gaussians in depth order are visible: compacted before the depth sort), so
  // that the gathers of all items are in flight together
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const int64_t s = base + k;
    c[k] = s < n ? order[s] : 0xFFFFFFFFu;
  }
#pragma unroll
  for (int k = 0; k < kSortItems; ++k)
    rc[k] = c[k] != 0xFFFFFFFFu ? rect[c[k]] : make_int4(0, 0, 0, 0);
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    uint32_t v = 0;
    const int4 r = rc[k];
    if (r.z > r.x) {
      const int gx0 = r.x / gw, gx1 = (r.z - 1) / gw + 1, gy0 = r.y / gh, gy1 = (r.w - 1) / gh + 1;
      v = (uint32_t)((gx1 - gx0) * (gy1 - gy0));
      atomicAdd(&D[gy0 * GXp1 + gx0], 1);
      atomicAdd(&D[gy0 * GXp1 + gx1], -1);
      atomicAdd(&D[gy1 * GXp1 + gx0], -1);
      atomicAdd(&D[gy1 * GXp1 + gx1], 1);
    }
    c[k] = v;
    sum += v;
  }
  uint64_t tile_total = 0;
  uint64_t run = block_excl_scan<uint64_t>(sum, tmp, &tile_total);
  if (threadIdx.x < 32) {
    const uint64_t pre = lookback64_warp(status, tile, tile_total, err);
    if (threadIdx.x == 0) s_prefix = pre;
  }
  __syncthreads();
  run += s_prefix;
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    if (base + k < n) offsets[base + k] = run;
    run += c[k];
  }
  if (base < n && base + kSortItems >= n) *total = (int64_t)run;  // the thread holding item n-1
  if (dslices) {
    int32_t* out = dslices + (size_t)tile * cells;
    for (int k = threadIdx.x; k < cells; k += kSortThreads) out[k] = sD[k];
  }
}

// Sums the tiles' difference slices per cell into `dsum` (zeroed before): blockIdx.y takes every
// gridDim.y-th tile, so many loads are in flight per cell.
__global__ void k_group_reduce(const int32_t* __restrict__ dslices,
                               const int64_t* __restrict__ visible, int cells,
                               int32_t* __restrict__ dsum) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cells) return;
  const int tiles = (int)((*visible + kSortTile - 1) / kSortTile);
  int32_t v = 0;
  for (int t = blockIdx.y; t < tiles; t += gridDim.y) v += dslices[(size_t)t * cells + c];
  if (v) atomicAdd(&dsum[c], v);
}

// From the difference array: per-group entry counts (2D prefix sum, in place), the group ranges
// (exclusive scan over row-major group ids) and the histograms of the group-id digits for the radix
// passes. One block; does nothing if the frame needs more entries than the capacity.
constexpr int kTableThreads = 1024;
__global__ void __launch_bounds__(kTableThreads) k_group_table(
    int32_t* __restrict__ Dg, int GX, int GY, int in_smem, const int64_t* __restrict__ total,
    int64_t cap, int passes, uint32_t* __restrict__ ranges, uint32_t* __restrict__ ghist) {
  extern __shared__ int32_t Ds[];
  __shared__ uint32_t h[kMaxPasses * kRadix];
  __shared__ uint32_t wsum[kTableThreads / 32];
  __shared__ uint32_t s_carry;
  if (*total > cap) return;
  const int GXp1 = GX + 1;
  int32_t* D = Dg;
  if (in_smem) {  // work on a shared copy of the cells
    for (int k = threadIdx.x; k < GXp1 * (GY + 1); k += kTableThreads) Ds[k] = Dg[k];
    D = Ds;
    __syncthreads();
  }
  for (int k = threadIdx.x; k < passes * kRadix; k += kTableThreads) h[k] = 0;
  // prefix along x (one thread per row), then along y (one thread per column)
  for (int y = threadIdx.x; y < GY; y += kTableThreads) {
    int32_t run = 0;
    for (int x = 0; x < GX; ++x) {
      run += D[y * GXp1 + x];
      D[y * GXp1 + x] = run;
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < GX; x += kTableThreads) {
    int32_t run = 0;
    for (int y = 0; y < GY; ++y) {
      run += D[y * GXp1 + x];
      D[y * GXp1 + x] = run;
    }
  }
  __syncthreads();
  // exclusive scan of the counts over g = y * GX + x, in chunks of the block's threads
  if (threadIdx.x == 0) s_carry = 0;
  const int G = GX * GY;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int g0 = 0; g0 < G; g0 += kTableThreads) {
    const int g = g0 + threadIdx.x;
    const uint32_t c = g < G ? (uint32_t)D[(g / GX) * GXp1 + (g % GX)] : 0u;
    const uint32_t incl = warp_incl_scan(c);
    __syncthreads();
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t add = s_carry;
    for (int w = 0; w < warp; ++w) add += wsum[w];
    const uint32_t start = add + incl - c;
    if (g < G) {
      ranges[2 * g] = c ? start : 0u;
      ranges[2 * g + 1] = c ? start + c : 0u;
      for (int p = 0; p < passes; ++p)
        if (c) atomicAdd(&h[p * kRadix + ((g >> (8 * p)) & 0xff)], c);
    }
    __syncthreads();
    if (threadIdx.x == kTableThreads - 1) s_carry = start + c;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < passes * kRadix; k += kTableThreads) ghist[k] = h[k];
}

// Duplicates each visible Gaussian once per overlapped group, in depth order. A warp handles 32
// consecutive Gaussians; their entries are contiguous in the output, so the warp writes them
// cooperatively (lane k of a round writes entry k), each lane locating its Gaussian by a binary
// search over the warp's prefix of counts.
__global__ void __launch_bounds__(256) k_emit(const int64_t* __restrict__ visible,
                                              const uint32_t* __restrict__ order,
                                              const int* __restrict__ radius,
                                              const int4* __restrict__ rect,
                                              const uint64_t* __restrict__ offsets,
                                              const int64_t* __restrict__ total, int64_t cap,
                                              int gw, int gh, int GX,
                                              uint32_t* __restrict__ gkeys,
                                              uint32_t* __restrict__ vals) {
  const int lane = threadIdx.x & 31;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = *visible;
  if (*total > cap || s - lane >= n) return;  // warp-uniform
  {
    uint32_t i = 0, cnt = 0;
    int gx0 = 0, gy0 = 0, gwn = 1;
    if (s < n) {
      i = order[s];
      if (radius[i] > 0) {
        const int4 r = rect[i];
        gx0 = r.x / gw;
        gy0 = r.y / gh;
        gwn = (r.z - 1) / gw - gx0 + 1;
        cnt = (uint32_t)(gwn * ((r.w - 1) / gh - gy0 + 1));
      }
    }
    const uint32_t incl = warp_incl_scan(cnt);
    const uint32_t warp_total = __shfl_sync(0xffffffffu, incl, 31);
    const uint64_t base = __shfl_sync(0xffffffffu, (s < n) ? offsets[s] : 0ull, 0);
    for (uint32_t k0 = 0; k0 < warp_total; k0 += 32) {
      const uint32_t k = k0 + lane;
      // smallest source lane whose inclusive prefix exceeds k
      int lo = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const uint32_t v = __shfl_sync(0xffffffffu, incl, lo + step - 1);
        if (v <= k) lo += step;
      }
      const uint32_t src_excl = __shfl_sync(0xffffffffu, incl - cnt, lo);
      const uint32_t src_i = __shfl_sync(0xffffffffu, i, lo);
      const int sx = __shfl_sync(0xffffffffu, gx0, lo), sy = __shfl_sync(0xffffffffu, gy0, lo);
      const int sw = __shfl_sync(0xffffffffu, gwn, lo);
      if (k < warp_total) {
        const int li = (int)(k - src_excl);
        // li / sw exactly: (li + 1/2) / sw is at least 1/(2 sw) away from an integer, far more
        // than the float rounding of the quotient (li < 2^24, sw <= 4096)
        const int qy = (int)(((float)li + 0.5f) * __frcp_rn((float)sw));
        const int qx = li - qy * sw;
        const uint64_t o = base + k;
        gkeys[o] = (uint32_t)((sy + qy) * GX + (sx + qx));
        vals[o] = src_i;
      }
    }
  }
}

// Masks and optional 64-bit keys of the sorted entries.
__global__ void k_finalize(const int64_t* __restrict__ total, int64_t cap,
                           const uint32_t* __restrict__ gkeys, const uint32_t* __restrict__ vals,
                           const Finalize fin) {
  const int64_t E = *total;
  if (E > cap) return;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x)
    entry_outputs(fin, (uint32_t)e, gkeys[e], vals[e]);
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Workspace: the ping-pong buffers, then one region that is cleared at the start of every call
// (digit histograms, look-back status words, tile tickets).
struct WsLayout {
  size_t dkA, dkB, dvA, dvB, offs, gkA, gkB, gvB, dslices;
  size_t zero_begin, hist_d, hist_g, stat_d, stat_g, stat_o, stat_c, tickets, dsum, visible,
      zero_end;
  int nb_c, nb_d, nb_g, nb_o, cells;
  bool sliced;  // the difference array fits in shared memory: per-tile slices
  size_t total;
};

constexpr int kMaxSmemCells = 11776;  // 46 KB of int32 difference cells per tile

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
  L.nb_d = (int)std::max<int64_t>(1, div_up(n, kSortThreads * kDepthItems));
  L.nb_g = (int)std::max<int64_t>(1, div_up(cap, kSortThreads * kGidItems));
  L.nb_o = L.nb_c;
  const int gpasses = std::max(1, div_up(group_bits(G), kRadixBits));
  L.dkA = take(4 * (size_t)n);
  L.dkB = take(4 * (size_t)n);
  L.dvA = take(4 * (size_t)n);
  L.dvB = take(4 * (size_t)n);
  L.offs = take(8 * (size_t)n);
  L.gkA = take(4 * (size_t)cap);
  L.gkB = take(4 * (size_t)cap);
  L.gvB = take(4 * (size_t)cap);
  L.cells = (GX + 1) * (GY + 1);
  L.sliced = L.cells <= kMaxSmemCells;
  L.dslices = take(L.sliced ? 4 * (size_t)L.nb_o * L.cells : 0);
  L.zero_begin = off;
  L.hist_d = take(4 * 4 * kRadix);
  L.hist_g = take(4 * (size_t)kMaxPasses * kRadix);
  L.stat_d = take(4 * (size_t)4 * L.nb_d * kRadix);
  L.stat_g = take(4 * (size_t)gpasses * L.nb_g * kRadix);
  L.stat_o = take(8 * (size_t)L.nb_o);
  L.stat_c = take(8 * (size_t)L.nb_c);
  L.tickets = take(4 * (4 + kMaxPasses + 2));
  L.visible = take(8);
  L.dsum = take(4 * (size_t)L.cells);
  L.zero_end = off;
  L.total = off;
  return L;
}

}  // namespace

size_t bin_sort_workspace_bytes(int64_t n, int64_t capacity, int GX, int GY) {
  return layout(n, capacity, GX, GY).total;
}

tgs_status launch_bin_sort(const tgs_projected& p, int64_t n64, int width, int height, int gw, int gh,
                           void* ws, size_t ws_bytes, const tgs_bins& b, cudaStream_t st) {
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
  const WsLayout L = layout(n64, cap, GX, GY);
  char* w = static_cast<char*>(ws);
  auto* dkA = reinterpret_cast<uint32_t*>(w + L.dkA);
  auto* dkB = reinterpret_cast<uint32_t*>(w + L.dkB);
  auto* dvA = reinterpret_cast<uint32_t*>(w + L.dvA);
  auto* dvB = reinterpret_cast<uint32_t*>(w + L.dvB);
  auto* offs = reinterpret_cast<uint64_t*>(w + L.offs);
  auto* gkA = reinterpret_cast<uint32_t*>(w + L.gkA);
  auto* gkB = reinterpret_cast<uint32_t*>(w + L.gkB);
  auto* gvB = reinterpret_cast<uint32_t*>(w + L.gvB);
  auto* hist_d = reinterpret_cast<uint32_t*>(w + L.hist_d);
  auto* hist_g = reinterpret_cast<uint32_t*>(w + L.hist_g);
  auto* stat_d = reinterpret_cast<uint32_t*>(w + L.stat_d);
  auto* stat_g = reinterpret_cast<uint32_t*>(w + L.stat_g);
  auto* stat_o = reinterpret_cast<uint64_t*>(w + L.stat_o);
  auto* tickets = reinterpret_cast<int*>(w + L.tickets);
  auto* dslices = L.sliced ? reinterpret_cast<int32_t*>(w + L.dslices) : nullptr;
  auto* dsum = reinterpret_cast<int32_t*>(w + L.dsum);
  const int4* rect = reinterpret_cast<const int4*>(p.rect);
  int32_t* err = device_error_word();
  TGS_CUDA(cudaMemsetAsync(w + L.zero_begin, 0, L.zero_end - L.zero_begin, st));

  // 1. depth order of the visible Gaussians: compacted keys + digit histograms, then four
  //    single-kernel radix passes over the visible count
  auto* visible = reinterpret_cast<int64_t*>(w + L.visible);
  auto* stat_c = reinterpret_cast<uint64_t*>(w + L.stat_c);
  k_depth_keys<<<L.nb_c, kSortThreads, 0, st>>>(n, p.radius, p.depth, dkA, dvA, visible, hist_d,
                                                stat_c, tickets + 4 + kMaxPasses + 1, err);
  TGS_CHECK_LAUNCH("k_depth_keys");
  const Finalize fin{rect, p.depth, gw, gh, GX, b.masks, b.keys};
  for (int pass = 0; pass < 4; ++pass) {
    const bool odd = pass & 1;
    k_onesweep<kDepthItems><<<L.nb_d, kSortThreads, 0, st>>>(
        odd ? dkB : dkA, odd ? dvB : dvA, odd ? dkA : dkB, odd ? dvA : dvB, visible, 0, n,
        8 * pass, hist_d + pass * kRadix, stat_d + (size_t)pass * L.nb_d * kRadix, tickets + pass,
        err);
    TGS_CHECK_LAUNCH("k_onesweep");
  }
  const uint32_t* order = dvA;  // after an even number of passes

  // 2. exclusive prefix of the group counts in depth order (total = needed entries) and the
  //    per-group entry counts -> group ranges and group-id digit histograms
  const int passes = div_up(group_bits(G), kRadixBits);
  k_group_offsets<<<L.nb_o, kSortThreads, L.sliced ? 4 * L.cells : 0, st>>>(
      visible, order, p.radius, rect, gw, gh, GX + 1, L.cells, offs, b.num_entries, dslices, dsum, stat_o,
      tickets + 4 + kMaxPasses, err);
  TGS_CHECK_LAUNCH("k_group_offsets");
  if (cap == 0) return TGS_OK;
  if (L.sliced) {
    const int tiles = div_up(n, kSortTile);
    k_group_reduce<<<dim3(div_up(L.cells, 256), std::min(tiles, 32)), 256, 0, st>>>(
        dslices, visible, L.cells, dsum);
    TGS_CHECK_LAUNCH("k_group_reduce");
  }
  // the attribute is the kernel's largest request, not this call's: CUDA graphs captured for other
  // image sizes launch the same function with their own sizes
  const int table_smem = L.sliced ? 4 * L.cells : 0;
  TGS_CUDA(cudaFuncSetAttribute(k_group_table, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                4 * kMaxSmemCells));
  k_group_table<<<1, kTableThreads, table_smem, st>>>(
      dsum, GX, GY, L.sliced ? 1 : 0, b.num_entries, cap, passes, b.ranges, hist_g);
  TGS_CHECK_LAUNCH("k_group_table");

  // 3. duplicate per overlapped group in depth order. The buffers are arranged so that the sorted
  //    Gaussian indices end in b.vals after an odd or even number of radix passes.
  uint32_t* ek = (passes & 1) ? gkB : gkA;
  uint32_t* ev = (passes & 1) ? gvB : b.vals;
  uint32_t* ok = (passes & 1) ? gkA : gkB;
  uint32_t* ov = (passes & 1) ? b.vals : gvB;
  k_emit<<<div_up(n, 256), 256, 0, st>>>(visible, order, p.radius, rect, offs, b.num_entries, cap, gw, gh,
                                          GX, ek, ev);
  TGS_CHECK_LAUNCH("k_emit");

  // 4. stable sort by group id
  const uint32_t* gk = ek;
  for (int pass = 0; pass < passes; ++pass) {
    const bool odd = pass & 1;
    k_onesweep<kGidItems><<<L.nb_g, kSortThreads, 0, st>>>(
        odd ? ok : ek, odd ? ov : ev, odd ? ek : ok, odd ? ev : ov, b.num_entries, 0, cap,
        8 * pass, hist_g + pass * kRadix, stat_g + (size_t)pass * L.nb_g * kRadix, tickets + 4 + pass,
        err);
    TGS_CHECK_LAUNCH("k_onesweep");
    gk = odd ? ek : ok;
  }

  // 5. masks and the optional 64-bit keys
  const int fin_blocks = std::max(1, std::min(div_up(cap, 256), 152 * 16));
  k_finalize<<<fin_blocks, 256, 0, st>>>(b.num_entries, cap, gk, b.vals, fin);
  TGS_CHECK_LAUNCH("k_finalize");
  return TGS_OK;
}

}  // namespace tgs
