// Plain FP32 CUDA-core rasterizer (Section 2 "Rasterization": one CTA per tile, one thread per
// pixel, all pixels of the tile walk the same depth-sorted list in shared-memory batches, with
// pruning and early termination). With group_w x group_h > 1 the CTA covers a tile group
// (Section 4.4.2) and each thread owns the same local pixel in several tiles; a list entry is used
// by a tile only if its mask bit is set. This is the baseline the tensor-core path is measured
// against, and the 1e-4 parity path.
#include <algorithm>

#include "tgs_internal.cuh"

namespace tgs {
namespace {

constexpr int kBatch = 256;

struct Pix {
  float T, r, g, b;
  int last;
  bool done;
};

template <int PPT, bool COUNT>
__global__ void __launch_bounds__(1024) k_raster_fp32(
    const uint32_t* __restrict__ ranges, const uint32_t* __restrict__ vals,
    const uint16_t* __restrict__ masks, const float2* __restrict__ mean2d,
    const float4* __restrict__ conic_opacity, const float* __restrict__ rgb, int width, int height,
    int gw, int gh, int GX, float3 bg, float* __restrict__ out_rgb, float* __restrict__ out_T,
    int* __restrict__ n_contrib, unsigned long long* __restrict__ counters) {
  __shared__ float2 s_xy[kBatch];
  __shared__ float4 s_co[kBatch];  // Cholesky factor of the conic (l11, l12, l22), opacity
  __shared__ float3 s_rgb[kBatch];
  __shared__ uint16_t s_mask[kBatch];

  const int gid = blockIdx.x;
  const int gx = gid % GX, gy = gid / GX;
  const int local = threadIdx.x & 255;           // pixel inside its tile
  const int tiles_per_pass = blockDim.x >> 8;    // tiles covered by one thread pass
  const int lx = local & 15, ly = local >> 4;

  int tile[PPT], px[PPT], py[PPT];
  Pix st[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    tile[k] = (threadIdx.x >> 8) + k * tiles_per_pass;
    const int tx = gx * gw + tile[k] % gw, ty = gy * gh + tile[k] / gw;
    px[k] = tx * kTile + lx;
    py[k] = ty * kTile + ly;
    const bool inside = tile[k] < gw * gh && px[k] < width && py[k] < height;
    st[k] = Pix{1.f, 0.f, 0.f, 0.f, 0, !inside};
  }

  const uint32_t start = ranges[2 * gid], end = ranges[2 * gid + 1];
  unsigned long long evaluated = 0, passing = 0, slots = 0;
  for (uint32_t base = start; base < end; base += kBatch) {
    bool all_done = true;
#pragma unroll
    for (int k = 0; k < PPT; ++k) all_done &= st[k].done;
    if (__syncthreads_count(!all_done) == 0) break;
    const int cnt = (int)min((uint32_t)kBatch, end - base);
    if (threadIdx.x < cnt) {
      const uint32_t e = base + threadIdx.x;
      const uint32_t i = vals[e];
      s_mask[threadIdx.x] = masks[e];
      s_xy[threadIdx.x] = mean2d[i];
      const float4 co = conic_opacity[i];
      const float3 L = conic_factor(co.x, co.y, co.z);
      s_co[threadIdx.x] = make_float4(L.x, L.y, L.z, co.w);
      s_rgb[threadIdx.x] = make_float3(rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2]);
    }
    __syncthreads();
    if (COUNT) slots += (unsigned long long)cnt * PPT;
    for (int j = 0; j < cnt; ++j) {
      const uint32_t m = s_mask[j];
      const float2 xy = s_xy[j];
      const float4 co = s_co[j];
      const int pos = (int)(base - start) + j + 1;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        if (!((m >> tile[k]) & 1u) || st[k].done) continue;
        if (COUNT) ++evaluated;
        const float dx = __fsub_rn((float)px[k], xy.x), dy = __fsub_rn((float)py[k], xy.y);
        const float power = power_fp32(make_float3(co.x, co.y, co.z), dx, dy);
        const float alpha = fminf(kAlphaMax, __fmul_rn(co.w, ex2(__fmul_rn(power, kLog2e))));
        if (alpha < kAlphaMin) continue;
        if (COUNT) ++passing;
        const float Tn = __fmul_rn(st[k].T, __fsub_rn(1.f, alpha));
        if (Tn < kTMin) {
          st[k].done = true;
          continue;
        }
        const float w = alpha * st[k].T;
        const float3 c = s_rgb[j];
        st[k].r += c.x * w;
        st[k].g += c.y * w;
        st[k].b += c.z * w;
        st[k].T = Tn;
        st[k].last = pos;
      }
    }
  }
  const size_t HW = (size_t)width * height;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    if (tile[k] >= gw * gh || px[k] >= width || py[k] >= height) continue;
    const size_t p = (size_t)py[k] * width + px[k];
    out_rgb[p] = st[k].r + st[k].T * bg.x;
    out_rgb[HW + p] = st[k].g + st[k].T * bg.y;
    out_rgb[2 * HW + p] = st[k].b + st[k].T * bg.z;
    out_T[p] = st[k].T;
    if (n_contrib) n_contrib[p] = st[k].last;
  }
  if (COUNT) {
    for (int o = 16; o > 0; o >>= 1) {
      evaluated += __shfl_xor_sync(0xffffffffu, evaluated, o);
      passing += __shfl_xor_sync(0xffffffffu, passing, o);
      slots += __shfl_xor_sync(0xffffffffu, slots, o);
    }
    if ((threadIdx.x & 31) == 0) {
      if (evaluated) atomicAdd(counters, evaluated);
      if (passing) atomicAdd(counters + 1, passing);
      if (slots) atomicAdd(counters + 2, slots);
    }
  }
}

template <int PPT>
tgs_status launch_ppt(int blocks, int threads, bool count, const tgs_projected& p, const tgs_bins& b,
                      int width, int height, int gw, int gh, int GX, float3 bg, float* out_rgb,
                      float* out_T, int32_t* n_contrib, unsigned long long* counters,
                      cudaStream_t st) {
  auto* m2 = reinterpret_cast<const float2*>(p.mean2d);
  auto* co = reinterpret_cast<const float4*>(p.conic_opacity);
  if (count)
    k_raster_fp32<PPT, true><<<blocks, threads, 0, st>>>(b.ranges, b.vals, b.masks, m2, co, p.rgb, width,
                                                         height, gw, gh, GX, bg, out_rgb, out_T,
                                                         n_contrib, counters);
  else
    k_raster_fp32<PPT, false><<<blocks, threads, 0, st>>>(b.ranges, b.vals, b.masks, m2, co, p.rgb, width,
                                                          height, gw, gh, GX, bg, out_rgb, out_T,
                                                          n_contrib, counters);
  TGS_CHECK_LAUNCH("k_raster_fp32");
  return TGS_OK;
}

}  // namespace

tgs_status launch_raster_fp32(const tgs_projected& p, const tgs_bins& b, int width, int height,
                              int gw, int gh, const tgs_raster_opts& o, float* out_rgb, float* out_T,
                              int32_t* n_contrib, cudaStream_t st) {
  if (((uintptr_t)p.mean2d & 7) || ((uintptr_t)p.conic_opacity & 15))
    return set_error("mean2d needs 8-byte and conic_opacity 16-byte alignment"), TGS_ERR_INVALID_ARGUMENT;
  const int TX = div_up(width, kTile), TY = div_up(height, kTile);
  const int GX = div_up(TX, gw), GY = div_up(TY, gh);
  const int tiles = gw * gh;
  const int threads = 256 * std::min(tiles, 4);
  const int ppt = div_up(tiles, threads / 256);
  const float3 bg = make_float3(o.bg[0], o.bg[1], o.bg[2]);
  auto* counters = reinterpret_cast<unsigned long long*>(o.counters);
  const bool count = counters != nullptr;
  const int blocks = GX * GY;
  switch (ppt) {
    case 1: return launch_ppt<1>(blocks, threads, count, p, b, width, height, gw, gh, GX, bg, out_rgb, out_T, n_contrib, counters, st);
    case 2: return launch_ppt<2>(blocks, threads, count, p, b, width, height, gw, gh, GX, bg, out_rgb, out_T, n_contrib, counters, st);
    case 3: return launch_ppt<3>(blocks, threads, count, p, b, width, height, gw, gh, GX, bg, out_rgb, out_T, n_contrib, counters, st);
    default: return launch_ppt<4>(blocks, threads, count, p, b, width, height, gw, gh, GX, bg, out_rgb, out_T, n_contrib, counters, st);
  }
}

}  // namespace tgs
