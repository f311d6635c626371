// Backward of the blend (Section 2 Eqs. power_d..blend differentiated by the chain rule; the paper
// trains FP16 and FP32 Gaussian models, Section 3.2.1, but prints no backward pass).
//
// For a pixel whose forward blended entries i = 1..m with alpha_i and T_i (T_1 = 1), colour
// C = sum_i alpha_i T_i c_i + T_final bg. Walking the pixel's list backwards from its last blended
// entry (n_contrib), T_i = T_{i+1} / (1 - alpha_i) is recovered from the stored final T (no per-entry
// state is kept by the forward), and with B the normalized colour behind entry i (B = bg after the
// last entry, then B <- alpha_i c_i + (1 - alpha_i) B):
//   dL/dc_i = alpha_i T_i G,  dL/dalpha_i = T_i G . (c_i - B),
//   alpha = o e^power unless clamped at 0.99 (then no gradient to o and power),
//   dpower/d(a, b, c) = (-dx^2/2, -dx dy, -dy^2/2), dpower/dmu' = (a dx + b dy, b dx + c dy).
// The per-entry alpha is recomputed with the same FP32 operation sequence as the FP32 forward, so
// every skip decision is replayed exactly. One CTA per tile group (as the forward); per entry the
// gradient contributions of the CTA's pixels are reduced per warp, then added with one atomic per
// warp and component.
#include <algorithm>

#include "tgs_internal.cuh"

namespace tgs {
namespace {

constexpr int kBatch = 256;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int PPT>
__global__ void __launch_bounds__(1024) k_raster_bwd(
    const uint32_t* __restrict__ ranges, const uint32_t* __restrict__ vals,
    const uint16_t* __restrict__ masks, const float2* __restrict__ mean2d,
    const float4* __restrict__ conic_opacity, const float* __restrict__ rgb, int width, int height,
    int gw, int gh, int GX, float3 bg, const float* __restrict__ out_T,
    const int* __restrict__ n_contrib, const float* __restrict__ grad_rgb,
    float* __restrict__ g_mean2d, float* __restrict__ g_co, float* __restrict__ g_rgb) {
  __shared__ float2 s_xy[kBatch];
  __shared__ float4 s_co[kBatch];
  __shared__ float4 s_L[kBatch];  // Cholesky factor of the conic (same forward arithmetic)
  __shared__ float3 s_rgb[kBatch];
  __shared__ uint16_t s_mask[kBatch];
  __shared__ uint32_t s_idx[kBatch];
  __shared__ int s_max_last;

  const int gid = blockIdx.x;
  const int gx = gid % GX, gy = gid / GX;
  const int local = threadIdx.x & 255;
  const int tiles_per_pass = blockDim.x >> 8;
  const int lx = local & 15, ly = local >> 4;
  const size_t HW = (size_t)width * height;

  int tile[PPT], last[PPT];
  float px[PPT], py[PPT], T[PPT];
  float3 G[PPT], B[PPT];
  int my_max = 0;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    tile[k] = (threadIdx.x >> 8) + k * tiles_per_pass;
    const int tx = gx * gw + tile[k] % gw, ty = gy * gh + tile[k] / gw;
    const int X = tx * kTile + lx, Y = ty * kTile + ly;
    px[k] = (float)X;
    py[k] = (float)Y;
    const bool inside = tile[k] < gw * gh && X < width && Y < height;
    last[k] = 0;
    T[k] = 1.f;
    G[k] = make_float3(0.f, 0.f, 0.f);
    B[k] = bg;
    if (inside) {
      const size_t p = (size_t)Y * width + X;
      last[k] = n_contrib[p];
      T[k] = out_T[p];
      G[k] = make_float3(grad_rgb[p], grad_rgb[HW + p], grad_rgb[2 * HW + p]);
    }
    my_max = max(my_max, last[k]);
  }
  if (threadIdx.x == 0) s_max_last = 0;
  __syncthreads();
  if (my_max) atomicMax(&s_max_last, my_max);
  __syncthreads();
  const int max_last = s_max_last;
  const uint32_t start = ranges[2 * gid];

  for (int hi = max_last; hi > 0; hi -= kBatch) {
    const int lo = max(0, hi - kBatch), cnt = hi - lo;
    __syncthreads();
    if (threadIdx.x < cnt) {
      const uint32_t e = start + lo + threadIdx.x;
      const uint32_t i = vals[e];
      s_idx[threadIdx.x] = i;
      s_mask[threadIdx.x] = masks[e];
      s_xy[threadIdx.x] = mean2d[i];
      const float4 co = conic_opacity[i];
      const float3 L = conic_factor(co.x, co.y, co.z);
      s_co[threadIdx.x] = co;
      s_L[threadIdx.x] = make_float4(L.x, L.y, L.z, 0.f);
      s_rgb[threadIdx.x] = make_float3(rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2]);
    }
    __syncthreads();
    for (int j = cnt - 1; j >= 0; --j) {
      const int pos = lo + j + 1;
      const uint32_t m = s_mask[j];
      const float2 xy = s_xy[j];
      const float4 co = s_co[j];
      const float4 Lf = s_L[j];
      const float3 L = make_float3(Lf.x, Lf.y, Lf.z);
      const float3 c = s_rgb[j];
      float gmx = 0.f, gmy = 0.f, ga = 0.f, gb = 0.f, gc = 0.f, go = 0.f, gr = 0.f, gg = 0.f,
            gbl = 0.f;
      bool any = false;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        if (pos > last[k] || !((m >> tile[k]) & 1u)) continue;
        const float dx = __fsub_rn(px[k], xy.x), dy = __fsub_rn(py[k], xy.y);
        const float power = power_fp32(L, dx, dy);
        const float ep = ex2(__fmul_rn(power, kLog2e));
        const float oe = __fmul_rn(co.w, ep);
        const float alpha = fminf(kAlphaMax, oe);
        if (alpha < kAlphaMin) continue;
        any = true;
        T[k] = T[k] / (1.f - alpha);  // T_i from T_{i+1}
        const float w = alpha * T[k];
        gr += w * G[k].x;
        gg += w * G[k].y;
        gbl += w * G[k].z;
        const float dLda =
            T[k] * (G[k].x * (c.x - B[k].x) + G[k].y * (c.y - B[k].y) + G[k].z * (c.z - B[k].z));
        B[k].x = alpha * c.x + (1.f - alpha) * B[k].x;
        B[k].y = alpha * c.y + (1.f - alpha) * B[k].y;
        B[k].z = alpha * c.z + (1.f - alpha) * B[k].z;
        if (oe <= kAlphaMax) {
          const float dLdp = dLda * alpha;
          go += dLda * ep;
          ga += dLdp * (-0.5f * dx * dx);
          gb += dLdp * (-dx * dy);
          gc += dLdp * (-0.5f * dy * dy);
          gmx += dLdp * (co.x * dx + co.y * dy);
          gmy += dLdp * (co.y * dx + co.z * dy);
        }
      }
      if (__any_sync(0xffffffffu, any)) {
        gmx = warp_sum(gmx); gmy = warp_sum(gmy);
        ga = warp_sum(ga); gb = warp_sum(gb); gc = warp_sum(gc); go = warp_sum(go);
        gr = warp_sum(gr); gg = warp_sum(gg); gbl = warp_sum(gbl);
        if ((threadIdx.x & 31) == 0) {
          const uint32_t i = s_idx[j];
          atomicAdd(&g_mean2d[2 * i], gmx);
          atomicAdd(&g_mean2d[2 * i + 1], gmy);
          atomicAdd(&g_co[4 * i], ga);
          atomicAdd(&g_co[4 * i + 1], gb);
          atomicAdd(&g_co[4 * i + 2], gc);
          atomicAdd(&g_co[4 * i + 3], go);
          atomicAdd(&g_rgb[3 * i], gr);
          atomicAdd(&g_rgb[3 * i + 1], gg);
          atomicAdd(&g_rgb[3 * i + 2], gbl);
        }
      }
    }
  }
}

}  // namespace

tgs_status launch_raster_backward(const tgs_projected& p, int64_t n, const tgs_bins& b, int width,
                                  int height, int gw, int gh, const tgs_raster_opts& o,
                                  const float* out_T, const int32_t* n_contrib, const float* grad_rgb,
                                  float* g_mean2d, float* g_conic_opacity, float* g_rgb,
                                  cudaStream_t st) {
  if (((uintptr_t)p.mean2d & 7) || ((uintptr_t)p.conic_opacity & 15))
    return set_error("mean2d needs 8-byte and conic_opacity 16-byte alignment"), TGS_ERR_INVALID_ARGUMENT;
  if (n > 0) {
    TGS_CUDA(cudaMemsetAsync(g_mean2d, 0, sizeof(float) * 2 * (size_t)n, st));
    TGS_CUDA(cudaMemsetAsync(g_conic_opacity, 0, sizeof(float) * 4 * (size_t)n, st));
    TGS_CUDA(cudaMemsetAsync(g_rgb, 0, sizeof(float) * 3 * (size_t)n, st));
  }
  const int TX = div_up(width, kTile), TY = div_up(height, kTile);
  const int GX = div_up(TX, gw), GY = div_up(TY, gh);
  const int tiles = gw * gh;
  const int threads = 256 * std::min(tiles, 4);
  const int ppt = div_up(tiles, threads / 256);
  const float3 bg = make_float3(o.bg[0], o.bg[1], o.bg[2]);
  auto* m2 = reinterpret_cast<const float2*>(p.mean2d);
  auto* co = reinterpret_cast<const float4*>(p.conic_opacity);
  const int blocks = GX * GY;
#define TGS_BWD(PPT)                                                                         \
  k_raster_bwd<PPT><<<blocks, threads, 0, st>>>(b.ranges, b.vals, b.masks, m2, co, p.rgb, width, \
                                                height, gw, gh, GX, bg, out_T, n_contrib,     \
                                                grad_rgb, g_mean2d, g_conic_opacity, g_rgb)
  switch (ppt) {
    case 1: TGS_BWD(1); break;
    case 2: TGS_BWD(2); break;
    case 3: TGS_BWD(3); break;
    default: TGS_BWD(4); break;
  }
#undef TGS_BWD
  TGS_CHECK_LAUNCH("k_raster_bwd");
  return TGS_OK;
}

}  // namespace tgs
