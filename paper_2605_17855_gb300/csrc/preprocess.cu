// Preprocess (Section 2 "Frustum culling" and "Feature computation"; Algorithm 1, the per-Gaussian
// screen-space attributes): cull, project the mean, EWA-project the covariance, invert it (the
// conic of Section 4.2.1), compute the 3-sigma radius and the overlapped tile range, and evaluate
// the SH colour. One thread per Gaussian; HBM-bound (about 236 B read + 56 B written per Gaussian
// at SH degree 3).
#include "tgs_internal.cuh"

namespace tgs {
namespace {

struct CamParams {
  int width, height;
  float fx, fy, cx, cy;
  float R[9], t[3], cam_pos[3];
  float near_z, limx, limy;
};

__device__ __forceinline__ void quat_rot_f32(float4 q, float Rq[9]) {
  const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
  Rq[0] = 1.f - 2.f * (y * y + z * z); Rq[1] = 2.f * (x * y - w * z); Rq[2] = 2.f * (x * z + w * y);
  Rq[3] = 2.f * (x * y + w * z); Rq[4] = 1.f - 2.f * (x * x + z * z); Rq[5] = 2.f * (y * z - w * x);
  Rq[6] = 2.f * (x * z - w * y); Rq[7] = 2.f * (y * z + w * x); Rq[8] = 1.f - 2.f * (x * x + y * y);
}

// 2D covariance (without dilation) as the Gram matrix of T3 = J W Rq S, the projected scaled axes:
// Sigma' = J W (Rq S)(Rq S)^T W^T J^T = T3 T3^T, and its determinant. By Lagrange's identity the
// determinant of a Gram matrix is |t0 x t1|^2 (t0, t1 the rows of T3), and with t_i = M j_i,
// M = S Rq^T W^T, the cofactor identity (M u) x (M v) = cof(M) (u x v) gives
// t0 x t1 = diag(s1 s2, s0 s2, s0 s1) Rq^T W^T (j0 x j1) (rotations are their own cofactors):
// products and rotations only, so the determinant keeps FP32 relative accuracy however thin the
// projected ellipse, where Sxx Syy - Sxy^2 would cancel.
__device__ __forceinline__ void cov2d_f32(const CamParams& c, float3 pc, float4 q, float3 s,
                                          float& cxx, float& cxy, float& cyy, float& det) {
  float Rq[9];
  quat_rot_f32(q, Rq);
  const float z = pc.z, iz = 1.f / z;
  const float xz = fminf(fmaxf(pc.x * iz, -c.limx), c.limx);
  const float yz = fminf(fmaxf(pc.y * iz, -c.limy), c.limy);
  const float j00 = c.fx * iz, j02 = -c.fx * xz * iz;
  const float j11 = c.fy * iz, j12 = -c.fy * yz * iz;
  float JW[6];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    JW[k] = j00 * c.R[k] + j02 * c.R[6 + k];
    JW[3 + k] = j11 * c.R[3 + k] + j12 * c.R[6 + k];
  }
  const float sv[3] = {s.x, s.y, s.z};
  float T0[3], T1[3];
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    T0[col] = (JW[0] * Rq[col] + JW[1] * Rq[3 + col] + JW[2] * Rq[6 + col]) * sv[col];
    T1[col] = (JW[3] * Rq[col] + JW[4] * Rq[3 + col] + JW[5] * Rq[6 + col]) * sv[col];
  }
  cxx = T0[0] * T0[0] + T0[1] * T0[1] + T0[2] * T0[2];
  cxy = T0[0] * T1[0] + T0[1] * T1[1] + T0[2] * T1[2];
  cyy = T1[0] * T1[0] + T1[1] * T1[1] + T1[2] * T1[2];
  // j0 = (j00, 0, j02), j1 = (0, j11, j12): j0 x j1 = (-j02 j11, -j00 j12, j00 j11)
  const float n[3] = {-j02 * j11, -j00 * j12, j00 * j11};
  float v[3], w[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) v[k] = c.R[k] * n[0] + c.R[3 + k] * n[1] + c.R[6 + k] * n[2];
#pragma unroll
  for (int k = 0; k < 3; ++k) w[k] = Rq[k] * v[0] + Rq[3 + k] * v[1] + Rq[6 + k] * v[2];
  const float d0 = s.y * s.z * w[0], d1 = s.x * s.z * w[1], d2 = s.x * s.y * w[2];
  det = d0 * d0 + d1 * d1 + d2 * d2;
}

// Real SH basis up to degree 3 (index l*l + m + l), Condon-Shortley phase kept in the real form.
template <int DEG>
__device__ __forceinline__ void sh_basis(float3 d, float (&Y)[16]) {
  const float x = d.x, y = d.y, z = d.z;
  Y[0] = 0.28209479177387814f;
  if (DEG >= 1) {
    const float k1 = 0.4886025119029199f;
    Y[1] = -k1 * y; Y[2] = k1 * z; Y[3] = -k1 * x;
  }
  if (DEG >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    const float a = 1.0925484305920792f, b = 0.31539156525252005f, c = 0.5462742152960396f;
    Y[4] = a * x * y; Y[5] = -a * y * z; Y[6] = b * (2.f * zz - xx - yy); Y[7] = -a * x * z;
    Y[8] = c * (xx - yy);
    if (DEG >= 3) {
      const float k3a = 0.5900435899266435f, k3b = 2.890611442640554f, k3c = 0.4570457994644658f,
                  k3d = 0.3731763325901154f, k3e = 1.445305721320277f;
      Y[9] = -k3a * y * (3.f * xx - yy);
      Y[10] = k3b * x * y * z;
      Y[11] = -k3c * y * (4.f * zz - xx - yy);
      Y[12] = k3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
      Y[13] = -k3c * x * (4.f * zz - xx - yy);
      Y[14] = k3e * z * (xx - yy);
      Y[15] = -k3a * x * (xx - 3.f * yy);
    }
  }
}

// Colour = sum_k sh[k] Y_k(d) + 0.5, clamped at 0. The coefficients are streamed (16-byte loads
// when the per-Gaussian block is a multiple of 16 bytes) and accumulated as they arrive.
template <int DEG>
__device__ __forceinline__ float3 sh_colour(const float* __restrict__ sp, float3 d) {
  constexpr int NC = (DEG + 1) * (DEG + 1);
  float Y[16];
  sh_basis<DEG>(d, Y);
  float acc[3] = {0.5f, 0.5f, 0.5f};
  if constexpr ((3 * NC) % 4 == 0) {
    const float4* sp4 = reinterpret_cast<const float4*>(sp);
#pragma unroll
    for (int k = 0; k < 3 * NC / 4; ++k) {
      const float4 v = __ldg(sp4 + k);
      const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int f = 4 * k + q;  // flattened (coefficient, channel)
        acc[f % 3] = fmaf(vv[q], Y[f / 3], acc[f % 3]);
      }
    }
  } else {
#pragma unroll
    for (int f = 0; f < 3 * NC; ++f) acc[f % 3] = fmaf(__ldg(sp + f), Y[f / 3], acc[f % 3]);
  }
  return make_float3(fmaxf(acc[0], 0.f), fmaxf(acc[1], 0.f), fmaxf(acc[2], 0.f));
}

__device__ __forceinline__ int64_t floor_div_tile(int64_t v) {
  return v >= 0 ? v / kTile : -((-v + kTile - 1) / kTile);
}

template <int DEG>
__global__ void __launch_bounds__(128, 8) k_preprocess(int n, const float* __restrict__ means,
                                                    const float* __restrict__ scales,
                                                    const float4* __restrict__ quats,
                                                    const float* __restrict__ opac,
                                                    const float* __restrict__ sh,
                                                    const __grid_constant__ CamParams c,
                                                    float2* __restrict__ mean2d,
                                                    float4* __restrict__ conic_opacity,
                                                    float* __restrict__ rgb,
                                                    float* __restrict__ depth,
                                                    int* __restrict__ radius,
                                                    int4* __restrict__ rect) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float m[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
  float3 pc;
  pc.x = c.R[0] * m[0] + c.R[1] * m[1] + c.R[2] * m[2] + c.t[0];
  pc.y = c.R[3] * m[0] + c.R[4] * m[1] + c.R[5] * m[2] + c.t[1];
  pc.z = c.R[6] * m[0] + c.R[7] * m[1] + c.R[8] * m[2] + c.t[2];

  float2 o_mean = make_float2(0.f, 0.f);
  float4 o_co = make_float4(0.f, 0.f, 0.f, 0.f);
  float3 o_rgb = make_float3(0.f, 0.f, 0.f);
  float o_depth = 0.f;
  int o_r = 0;
  int4 o_rect = make_int4(0, 0, 0, 0);

  if (pc.z > c.near_z) {
    const float4 q = quats[i];
    const float3 s = make_float3(scales[3 * i], scales[3 * i + 1], scales[3 * i + 2]);
    float cxx, cxy, cyy, det;
    cov2d_f32(c, pc, q, s, cxx, cxy, cyy, det);
    // dilation by 0.3 I: det(S + 0.3 I) = det S + 0.3 tr S + 0.09, a sum of non-negative terms
    det = det + 0.3f * (cxx + cyy) + 0.09f;
    cxx += 0.3f;
    cyy += 0.3f;
    const float ca = cyy / det, cb = -cxy / det, cc = cxx / det;
    if (det > 0.f) {
      const float mx = c.fx * pc.x / pc.z + c.cx;
      const float my = c.fy * pc.y / pc.z + c.cy;
      const float mid = 0.5f * (cxx + cyy);
      const float disc = fmaxf(0.1f, mid * mid - det);
      const float lmax = mid + sqrtf(disc);
      const float rf = fminf(ceilf(3.f * sqrtf(lmax)), 16777216.f);
      const int r = (int)rf;
      // pixel i lies in [m - r, m + r] iff ceil(m) - r <= i <= floor(m) + r
      const float mxc = fminf(fmaxf(mx, -1e9f), 1e9f), myc = fminf(fmaxf(my, -1e9f), 1e9f);
      const int64_t bx0 = (int64_t)ceilf(mxc) - r, bx1 = (int64_t)floorf(mxc) + r;
      const int64_t by0 = (int64_t)ceilf(myc) - r, by1 = (int64_t)floorf(myc) + r;
      const int64_t px0 = bx0 > 0 ? bx0 : 0, px1 = bx1 < c.width - 1 ? bx1 : c.width - 1;
      const int64_t py0 = by0 > 0 ? by0 : 0, py1 = by1 < c.height - 1 ? by1 : c.height - 1;
      if (px0 <= px1 && py0 <= py1) {
        o_rect = make_int4((int)floor_div_tile(px0), (int)floor_div_tile(py0),
                           (int)floor_div_tile(px1) + 1, (int)floor_div_tile(py1) + 1);
        o_r = r;
        o_mean = make_float2(mx, my);
        o_co = make_float4(ca, cb, cc, opac[i]);
        o_depth = pc.z;
        float3 d = make_float3(m[0] - c.cam_pos[0], m[1] - c.cam_pos[1], m[2] - c.cam_pos[2]);
        const float inv = 1.f / sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
        d.x *= inv; d.y *= inv; d.z *= inv;
        constexpr int NC = (DEG + 1) * (DEG + 1);
        o_rgb = sh_colour<DEG>(sh + (int64_t)i * 3 * NC, d);
      }
    }
  }
  radius[i] = o_r;
  if (o_r == 0) return;  // culled: no consumer reads the other outputs of this Gaussian
  mean2d[i] = o_mean;
  conic_opacity[i] = o_co;
  rgb[3 * i] = o_rgb.x;
  rgb[3 * i + 1] = o_rgb.y;
  rgb[3 * i + 2] = o_rgb.z;
  depth[i] = o_depth;
  rect[i] = o_rect;
}

}  // namespace

tgs_status launch_preprocess(const tgs_scene& s, const tgs_camera& cam, const tgs_projected& out,
                             cudaStream_t st) {
  CamParams c;
  c.width = cam.width; c.height = cam.height;
  c.fx = cam.fx; c.fy = cam.fy; c.cx = cam.cx; c.cy = cam.cy;
  for (int k = 0; k < 9; ++k) c.R[k] = cam.R[k];
  for (int k = 0; k < 3; ++k) { c.t[k] = cam.t[k]; c.cam_pos[k] = cam.cam_pos[k]; }
  c.near_z = cam.near_z;
  c.limx = 1.3f * 0.5f * (float)cam.width / cam.fx;
  c.limy = 1.3f * 0.5f * (float)cam.height / cam.fy;
  if (((uintptr_t)s.quats & 15) || ((uintptr_t)out.conic_opacity & 15) || ((uintptr_t)out.rect & 15) ||
      ((uintptr_t)out.mean2d & 7) || (s.sh_degree % 2 == 1 && ((uintptr_t)s.sh & 15))) {
    set_error("misaligned array (quats, conic_opacity, rect need 16 B; mean2d 8 B; sh 16 B)");
    return TGS_ERR_INVALID_ARGUMENT;
  }
  const int n = (int)s.n;
  const int threads = 128, blocks = div_up(n, threads);
  auto* q4 = reinterpret_cast<const float4*>(s.quats);
  auto* m2 = reinterpret_cast<float2*>(out.mean2d);
  auto* co = reinterpret_cast<float4*>(out.conic_opacity);
  auto* rc = reinterpret_cast<int4*>(out.rect);
  switch (s.sh_degree) {
    case 0: k_preprocess<0><<<blocks, threads, 0, st>>>(n, s.means, s.scales, q4, s.opacities, s.sh, c, m2, co, out.rgb, out.depth, out.radius, rc); break;
    case 1: k_preprocess<1><<<blocks, threads, 0, st>>>(n, s.means, s.scales, q4, s.opacities, s.sh, c, m2, co, out.rgb, out.depth, out.radius, rc); break;
    case 2: k_preprocess<2><<<blocks, threads, 0, st>>>(n, s.means, s.scales, q4, s.opacities, s.sh, c, m2, co, out.rgb, out.depth, out.radius, rc); break;
    default: k_preprocess<3><<<blocks, threads, 0, st>>>(n, s.means, s.scales, q4, s.opacities, s.sh, c, m2, co, out.rgb, out.depth, out.radius, rc); break;
  }
  TGS_CHECK_LAUNCH("k_preprocess");
  return TGS_OK;
}

}  // namespace tgs
