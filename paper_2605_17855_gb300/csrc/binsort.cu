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
//   depth keys -> radix(depth) -> per-Gaussian group counts -> exclusive scan (u64) -> emit
//   (gid, index) -> radix(gid) -> finalize (64-bit keys, masks from the tile ranges, group ranges).
#include <algorithm>

#include "tgs_internal.cuh"

namespace tgs {
namespace {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;  // 8 warps
constexpr int kSortItems = 16;     // per thread
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 items per block
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t live_count(const int64_t* count_dev, int64_t count_host,
                                              int64_t cap) {
  if (!count_dev) return count_host;
  const int64_t c = *count_dev;
  return (c < 0 || c > cap) ? 0 : c;
}

// ---------------------------------------------------------------------------------------------
// Exclusive scan (multi-kernel; no inter-block waiting).
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

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_block(const T* in, T* out, T* block_sums,
                                                             int64_t count, T* total) {
  __shared__ T warp_tot[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < count) ? in[base + k] : T(0);
    sum += v[k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T incl = warp_incl_scan(sum);
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T w = lane < kScanThreads / 32 ? warp_tot[lane] : T(0);
    w = warp_incl_scan(w);
    if (lane < kScanThreads / 32) warp_tot[lane] = w;
  }
  __syncthreads();
  T run = incl - sum + (warp ? warp_tot[warp - 1] : T(0));
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < count) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == kScanThreads - 1) {
    if (block_sums) block_sums[blockIdx.x] = run;
    if (total) *total = run;
  }
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_add(T* out, const T* offs, int64_t count) {
  const T add = offs[blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int k = threadIdx.x; k < kScanTile; k += kScanThreads)
    if (base + k < count) out[base + k] += add;
}

template <typename T>
size_t scan_scratch_elems(int64_t count) {
  size_t s = 0;
  while (count > kScanTile) {
    count = div_up(count, kScanTile);
    s += count;
  }
  return s;
}

// In-place capable exclusive scan of `count` elements; writes the total to `total` if non-null.
template <typename T>
tgs_status scan_exclusive(const T* in, T* out, int64_t count, T* scratch, T* total,
                          cudaStream_t st) {
  if (count <= 0) {
    if (total) TGS_CUDA(cudaMemsetAsync(total, 0, sizeof(T), st));
    return TGS_OK;
  }
  const int blocks = div_up(count, kScanTile);
  if (blocks == 1) {
    k_scan_block<T><<<1, kScanThreads, 0, st>>>(in, out, nullptr, count, total);
    TGS_CHECK_LAUNCH("k_scan_block");
    return TGS_OK;
  }
  T* sums = scratch;
  k_scan_block<T><<<blocks, kScanThreads, 0, st>>>(in, out, sums, count, nullptr);
  TGS_CHECK_LAUNCH("k_scan_block");
  tgs_status s = scan_exclusive<T>(sums, sums, blocks, scratch + blocks, total, st);
  if (s != TGS_OK) return s;
  k_scan_add<T><<<blocks, kScanThreads, 0, st>>>(out, sums, count);
  TGS_CHECK_LAUNCH("k_scan_add");
  return TGS_OK;
}

// ---------------------------------------------------------------------------------------------
// One stable LSD radix pass (8-bit digit at `shift`) of (u32 key, u32 value) pairs.
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ keys,
                                                             const int64_t* count_dev,
                                                             int64_t count_host, int64_t cap,
                                                             int shift, uint32_t* __restrict__ hist,
                                                             int num_blocks) {
  __shared__ uint32_t h[kRadix];
  for (int k = threadIdx.x; k < kRadix; k += kSortThreads) h[k] = 0;
  __syncthreads();
  const int64_t count = live_count(count_dev, count_host, cap);
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  if (base < count) {
    for (int k = threadIdx.x; k < kSortTile; k += kSortThreads) {
      const int64_t i = base + k;
      if (i < count) atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1u);
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads)
    hist[(int64_t)d * num_blocks + blockIdx.x] = h[d];
}

// Stable scatter of one pass. Each warp ranks its 256 consecutive items by digit (match_any),
// warps are ordered, so the block's items get their stable position in digit order; they are staged
// in shared memory in that order and written out so that each digit's run is contiguous and the
// global stores of consecutive threads are consecutive.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, const int64_t* count_dev,
    int64_t count_host, int64_t cap, int shift, const uint32_t* __restrict__ offsets,
    int num_blocks) {
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t wcount[W][kRadix];  // per warp and digit: count, then exclusive offset
  __shared__ uint32_t dstart[kRadix];     // block-local start of each digit's run
  __shared__ uint32_t boff[kRadix];       // global start of this block's run of each digit
  __shared__ uint32_t warp_tot[kRadix / 32];
  __shared__ uint32_t skey[kSortTile], sval[kSortTile];
  const int64_t count = live_count(count_dev, count_host, cap);
  const int64_t block_base = (int64_t)blockIdx.x * kSortTile;
  if (block_base >= count) return;  // uniform per block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < W * kRadix; k += kSortThreads) (&wcount[0][0])[k] = 0;
  __syncthreads();
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
  int dig[kSortItems];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t i = block_base + (int64_t)warp * (32 * kSortItems) + r * 32 + lane;
    const bool valid = i < count;
    key[r] = valid ? keys_in[i] : 0u;
    val[r] = valid ? vals_in[i] : 0u;
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
  // per digit: exclusive offsets over warps and the block total; then an exclusive scan of the
  // totals over digits (one thread per digit)
  static_assert(kSortThreads >= kRadix, "one thread per digit");
  uint32_t total = 0;
  if (threadIdx.x < kRadix) {
    const int d = threadIdx.x;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint32_t c = wcount[w][d];
      wcount[w][d] = total;
      total += c;
    }
    boff[d] = offsets[(int64_t)d * num_blocks + blockIdx.x];
    uint32_t incl = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) warp_tot[warp] = incl;
    total = incl - total;  // exclusive within the warp
  }
  __syncthreads();
  if (threadIdx.x < kRadix) {
    uint32_t add = 0;
    for (int w = 0; w < warp; ++w) add += warp_tot[w];
    dstart[threadIdx.x] = total + add;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int d = dig[r];
    if (d < kRadix) {
      const uint32_t p = dstart[d] + wcount[warp][d] + rank[r];
      skey[p] = key[r];
      sval[p] = val[r];
    }
  }
  __syncthreads();
  const int nvalid = (int)min((int64_t)kSortTile, count - block_base);
  for (int i = threadIdx.x; i < nvalid; i += kSortThreads) {
    const uint32_t k = skey[i];
    const int d = (int)((k >> shift) & (kRadix - 1));
    const uint32_t pos = boff[d] + (uint32_t)i - dstart[d];
    keys_out[pos] = k;
    vals_out[pos] = sval[i];
  }
}

// Sorts (keys, vals) by the low `bits` bits; ping-pongs between the A and B buffers. Returns the
// buffer index (0 = A, 1 = B) holding the result.
tgs_status radix_sort(uint32_t* kA, uint32_t* vA, uint32_t* kB, uint32_t* vB,
                      const int64_t* count_dev, int64_t count_host, int64_t cap, int bits,
                      uint32_t* hist, uint32_t* scan_scratch, cudaStream_t st, int* result_in) {
  const int64_t max_items = count_dev ? cap : count_host;
  const int num_blocks = std::max(1, div_up(max_items, kSortTile));
  int cur = 0;
  for (int shift = 0; shift < bits; shift += kRadixBits) {
    const uint32_t* ki = cur ? kB : kA;
    const uint32_t* vi = cur ? vB : vA;
    uint32_t* ko = cur ? kA : kB;
    uint32_t* vo = cur ? vA : vB;
    k_radix_hist<<<num_blocks, kSortThreads, 0, st>>>(ki, count_dev, count_host, cap, shift, hist,
                                                      num_blocks);
    TGS_CHECK_LAUNCH("k_radix_hist");
    tgs_status s = scan_exclusive<uint32_t>(hist, hist, (int64_t)kRadix * num_blocks, scan_scratch,
                                            nullptr, st);
    if (s != TGS_OK) return s;
    k_radix_scatter<<<num_blocks, kSortThreads, 0, st>>>(ki, vi, ko, vo, count_dev, count_host, cap,
                                                         shift, hist, num_blocks);
    TGS_CHECK_LAUNCH("k_radix_scatter");
    cur ^= 1;
  }
  *result_in = cur;
  return TGS_OK;
}

// ---------------------------------------------------------------------------------------------
// Binning kernels.
__global__ void k_depth_keys(int n, const int* __restrict__ radius, const float* __restrict__ depth,
                             uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // depth > near_z > 0, so the IEEE bits of a visible depth are monotone in the depth;
  // culled Gaussians get the largest key and sort last
  keys[i] = radius[i] > 0 ? __float_as_uint(depth[i]) : 0xFFFFFFFFu;
  vals[i] = (uint32_t)i;
}

__global__ void k_group_counts(int n, const uint32_t* __restrict__ order,
                               const int* __restrict__ radius, const int4* __restrict__ rect,
                               int gw, int gh, uint64_t* __restrict__ counts) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint32_t i = order[s];
  uint64_t c = 0;
  if (radius[i] > 0) {
    const int4 r = rect[i];
    c = (uint64_t)((r.z - 1) / gw - r.x / gw + 1) * (uint64_t)((r.w - 1) / gh - r.y / gh + 1);
  }
  counts[s] = c;
}

// Duplicates each visible Gaussian once per overlapped group, in depth order. A warp handles 32
// consecutive Gaussians; their entries are contiguous in the output, so the warp writes them
// cooperatively (lane k of a round writes entry k), each lane locating its Gaussian by a binary
// search over the warp's prefix of counts.
__global__ void __launch_bounds__(256) k_emit(int n, const uint32_t* __restrict__ order,
                                              const int* __restrict__ radius,
                                              const int4* __restrict__ rect,
                                              const uint64_t* __restrict__ offsets,
                                              const int64_t* __restrict__ total, int64_t cap,
                                              int gw, int gh, int GX, uint32_t* __restrict__ gkeys,
                                              uint32_t* __restrict__ vals) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  if (*total > cap) return;
  if ((s - lane) >= n) return;  // the whole warp is past the end
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
  // inclusive prefix of the counts over the warp
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
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
      const uint64_t o = base + k;
      gkeys[o] = (uint32_t)((sy + li / sw) * GX + (sx + li % sw));
      vals[o] = src_i;
    }
  }
}

__global__ void k_finalize(const int64_t* __restrict__ total, int64_t cap,
                           const uint32_t* __restrict__ gkeys, const uint32_t* __restrict__ vals,
                           const float* __restrict__ depth, const int4* __restrict__ rect, int gw,
                           int gh, int GX, uint64_t* __restrict__ keys64,
                           uint16_t* __restrict__ masks, uint32_t* __restrict__ ranges) {
  const int64_t E = *total;
  if (E > cap) return;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t g = gkeys[e];
    const uint32_t i = vals[e];
    if (keys64) keys64[e] = ((uint64_t)g << 32) | __float_as_uint(depth[i]);
    const int4 r = rect[i];
    const int gx = (int)(g % (uint32_t)GX), gy = (int)(g / (uint32_t)GX);
    uint32_t m = 0;
    for (int ty = 0; ty < gh; ++ty)
      for (int tx = 0; tx < gw; ++tx) {
        const int X = gx * gw + tx, Y = gy * gh + ty;
        if (X >= r.x && X < r.z && Y >= r.y && Y < r.w) m |= 1u << (ty * gw + tx);
      }
    masks[e] = (uint16_t)m;
    if (e == 0 || gkeys[e - 1] != g) ranges[2 * g] = (uint32_t)e;
    if (e == E - 1 || gkeys[e + 1] != g) ranges[2 * g + 1] = (uint32_t)(e + 1);
  }
}

struct WsLayout {
  size_t dkA, dkB, dvA, dvB, counts, gkA, gkB, gvB, hist, scan32, scan64, total;
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

WsLayout layout(int64_t n, int64_t cap) {
  WsLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  const int64_t nb = std::max<int64_t>(1, std::max(div_up(n, kSortTile), div_up(cap, kSortTile)));
  L.dkA = take(4 * (size_t)n);
  L.dkB = take(4 * (size_t)n);
  L.dvA = take(4 * (size_t)n);
  L.dvB = take(4 * (size_t)n);
  L.counts = take(8 * (size_t)n);
  L.gkA = take(4 * (size_t)cap);
  L.gkB = take(4 * (size_t)cap);
  L.gvB = take(4 * (size_t)cap);
  L.hist = take(4 * (size_t)kRadix * nb);
  L.scan32 = take(4 * scan_scratch_elems<uint32_t>((int64_t)kRadix * nb));
  L.scan64 = take(8 * scan_scratch_elems<uint64_t>(n));
  L.total = off;
  return L;
}

}  // namespace

size_t bin_sort_workspace_bytes(int64_t n, int64_t capacity, int num_groups) {
  (void)num_groups;
  return layout(n, capacity).total;
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
  const WsLayout L = layout(n64, cap);
  char* w = static_cast<char*>(ws);
  auto* dkA = reinterpret_cast<uint32_t*>(w + L.dkA);
  auto* dkB = reinterpret_cast<uint32_t*>(w + L.dkB);
  auto* dvA = reinterpret_cast<uint32_t*>(w + L.dvA);
  auto* dvB = reinterpret_cast<uint32_t*>(w + L.dvB);
  auto* counts = reinterpret_cast<uint64_t*>(w + L.counts);
  auto* gkA = reinterpret_cast<uint32_t*>(w + L.gkA);
  auto* gkB = reinterpret_cast<uint32_t*>(w + L.gkB);
  auto* gvB = reinterpret_cast<uint32_t*>(w + L.gvB);
  auto* hist = reinterpret_cast<uint32_t*>(w + L.hist);
  auto* scan32 = reinterpret_cast<uint32_t*>(w + L.scan32);
  auto* scan64 = reinterpret_cast<uint64_t*>(w + L.scan64);
  const int4* rect = reinterpret_cast<const int4*>(p.rect);
  const int threads = 256;

  // 1. depth order of the visible Gaussians (culled ones last)
  k_depth_keys<<<div_up(n, threads), threads, 0, st>>>(n, p.radius, p.depth, dkA, dvA);
  TGS_CHECK_LAUNCH("k_depth_keys");
  int where = 0;
  tgs_status s = radix_sort(dkA, dvA, dkB, dvB, nullptr, n, n, 32, hist, scan32, st, &where);
  if (s != TGS_OK) return s;
  const uint32_t* order = where ? dvB : dvA;

  // 2. group counts in depth order, exclusive scan, total = needed entries
  k_group_counts<<<div_up(n, threads), threads, 0, st>>>(n, order, p.radius, rect, gw, gh, counts);
  TGS_CHECK_LAUNCH("k_group_counts");
  s = scan_exclusive<uint64_t>(counts, counts, n, scan64, reinterpret_cast<uint64_t*>(b.num_entries), st);
  if (s != TGS_OK) return s;
  if (cap == 0) return TGS_OK;

  // 3. duplicate per overlapped group in depth order. The buffers are arranged so that the sorted
  //    Gaussian indices end in b.vals after an odd or even number of radix passes.
  int gbits = 0;
  while ((int64_t(1) << gbits) < G) ++gbits;
  const int passes = (gbits + kRadixBits - 1) / kRadixBits;
  uint32_t* ek = (passes & 1) ? gkB : gkA;
  uint32_t* ev = (passes & 1) ? gvB : b.vals;
  uint32_t* ok = (passes & 1) ? gkA : gkB;
  uint32_t* ov = (passes & 1) ? b.vals : gvB;
  k_emit<<<div_up(n, 256), 256, 0, st>>>(n, order, p.radius, rect, counts, b.num_entries, cap, gw, gh,
                                          GX, ek, ev);
  TGS_CHECK_LAUNCH("k_emit");

  // 4. stable sort by group id
  const uint32_t* gk = ek;
  if (passes > 0) {
    s = radix_sort(ek, ev, ok, ov, b.num_entries, 0, cap, gbits, hist, scan32, st, &where);
    if (s != TGS_OK) return s;
    gk = where ? ok : ek;
  }
  const uint32_t* gv = b.vals;

  // 5. 64-bit keys, masks, group ranges
  const int fin_blocks = std::max(1, std::min(div_up(cap, threads), 152 * 16));
  k_finalize<<<fin_blocks, threads, 0, st>>>(b.num_entries, cap, gk, gv, p.depth, rect, gw, gh, GX,
                                             b.keys, b.masks, b.ranges);
  TGS_CHECK_LAUNCH("k_finalize");
  return TGS_OK;
}

}  // namespace tgs
