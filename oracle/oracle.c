/* FP64 CPU oracle of the tile-based 3D Gaussian Splatting rasterizer with cross-tile grouping.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the benchmark's
 * CPU-baseline leg. The rendering library never links, loads or calls it; the two share no code.
 *
 * What it computes, in the order of the paper (TensorGS, "Accelerating 3D Gaussian Splatting using
 * Tensor Cores"):
 *   Section 2 "Frustum culling", "Feature computation": cull, project the mean, EWA-project the
 *     covariance, invert it (the conic of Section 4.2.1), find the tiles the splat's AABB overlaps,
 *     evaluate the SH colour.
 *   Section 4.4.2 / Algorithm 1: one entry per overlapped tile group with a tile-membership mask,
 *     sorted by (group ID, depth).
 *   Section 2 Eqs. power_d, power, alpha, blend, plus pruning and early termination: per pixel,
 *     walk the depth-ordered list of its tile (the group list filtered by the mask bit).
 *   The backward of that blend by the chain rule.
 * The paper prints no code; the power is evaluated in the scalar form of Eq. tensorgs_power_scalar
 * (no GEMM, no grouping shortcut): the method reaches this same result exactly (padding, Sec. 4.2.3;
 * grouping, Sec. 4.4.2), so this plain definition is the oracle.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - pixel (i, j) is sampled at image coordinates (i, j);
 *   - culling: camera-space z <= near_z culls; no side-plane cull beyond an empty tile range;
 *     the EWA Jacobian is taken at x/z, y/z clamped to +-1.3 tan(half FOV);
 *   - the projected covariance is dilated by 0.3 I before inversion;
 *   - radius r = ceil(3 sqrt(lambda_max)), lambda from the 2x2 eigenproblem with the discriminant
 *     floored at 0.1; the AABB is [mu - r, mu + r]^2 and a tile is overlapped iff one of its
 *     image pixels lies inside it (closed bounds);
 *   - SH: real spherical harmonics, degree <= 3, index l*l + m + l, Condon-Shortley phase kept in the
 *     real form; colour = sum + 0.5, clamped at 0 per channel;
 *   - tile membership (beyond the paper, whose Section 6 cites tighter splat footprints): a tile of
 *     the AABB's range stays in a splat's entry only if the splat's ellipse at the level where
 *     o e^power could reach 1/255 (plus slack) meets the tile's pixel-centre box; the test is a
 *     decision about which entries exist, so it is taken in FP32 with a fixed operation order
 *     (member_setup / member_row below), the precision of the kernels, and it is conservative:
 *     a dropped (splat, tile) pair is pruned at every pixel of the tile;
 *   - group IDs are row-major over groups; mask bit (ty - gy*gh)*gw + (tx - gx*gw);
 *     key = (gid << 32) | bits(float(depth)), ties broken by splat index;
 *   - alpha = min(0.99, o exp(power)); alpha < 1/255 skips; an entry whose T' = T (1 - alpha)
 *     falls below 1e-4 is not blended and ends the pixel; a power > 0 is skipped (never happens for
 *     a positive-definite conic in exact arithmetic; counted).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off (no FMA contraction, so x86 and Arm agree).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int32_t orc_num_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------------------------------------
 * Spherical harmonics (Section 2: colour from SH coefficients and the viewing direction).
 * Real SH built from the complex Y_l^m (with Condon-Shortley phase): m < 0 -> sqrt2 Im Y_l^|m|,
 * m = 0 -> Y_l^0, m > 0 -> sqrt2 Re Y_l^m, written as polynomials of the unit direction (x, y, z). */
void orc_sh_basis(const double d[3], double out[16]) {
  const double x = d[0], y = d[1], z = d[2];
  const double pi = 3.14159265358979323846;
  out[0] = 0.5 * sqrt(1.0 / pi);
  const double k1 = sqrt(3.0 / (4.0 * pi));
  out[1] = -k1 * y;
  out[2] = k1 * z;
  out[3] = -k1 * x;
  const double k2a = 0.5 * sqrt(15.0 / pi), k2b = 0.25 * sqrt(5.0 / pi), k2c = 0.25 * sqrt(15.0 / pi);
  out[4] = k2a * x * y;
  out[5] = -k2a * y * z;
  out[6] = k2b * (2.0 * z * z - x * x - y * y);
  out[7] = -k2a * x * z;
  out[8] = k2c * (x * x - y * y);
  const double k3a = 0.125 * sqrt(70.0 / pi), k3b = 0.5 * sqrt(105.0 / pi),
               k3c = 0.125 * sqrt(42.0 / pi), k3d = 0.25 * sqrt(7.0 / pi),
               k3e = 0.25 * sqrt(105.0 / pi);
  out[9] = -k3a * y * (3.0 * x * x - y * y);
  out[10] = k3b * x * y * z;
  out[11] = -k3c * y * (4.0 * z * z - x * x - y * y);
  out[12] = k3d * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
  out[13] = -k3c * x * (4.0 * z * z - x * x - y * y);
  out[14] = k3e * z * (x * x - y * y);
  out[15] = -k3a * x * (x * x - 3.0 * y * y);
}

/* Rotation matrix of the normalized quaternion (w, x, y, z), row-major. */
static void quat_to_rotation(const float* qf, double Rq[9]) {
  double w = qf[0], x = qf[1], y = qf[2], z = qf[3];
  const double nrm = sqrt(w * w + x * x + y * y + z * z);
  w /= nrm; x /= nrm; y /= nrm; z /= nrm;
  Rq[0] = 1.0 - 2.0 * (y * y + z * z); Rq[1] = 2.0 * (x * y - w * z); Rq[2] = 2.0 * (x * z + w * y);
  Rq[3] = 2.0 * (x * y + w * z); Rq[4] = 1.0 - 2.0 * (x * x + z * z); Rq[5] = 2.0 * (y * z - w * x);
  Rq[6] = 2.0 * (x * z - w * y); Rq[7] = 2.0 * (y * z + w * x); Rq[8] = 1.0 - 2.0 * (x * x + y * y);
}

static void to_camera(const orc_camera* cam, const float* m, double pc[3]) {
  for (int r = 0; r < 3; ++r)
    pc[r] = cam->R[3 * r + 0] * (double)m[0] + cam->R[3 * r + 1] * (double)m[1] +
            cam->R[3 * r + 2] * (double)m[2] + cam->t[r];
}

/* EWA projection of the 3D covariance Sigma = (Rq S)(Rq S)^T to the image plane:
 * Sigma' = J W Sigma W^T J^T with W the camera rotation and J the Jacobian of the perspective map
 * (u, v) = (fx x/z + cx, fy y/z + cy) at the (clamped) camera-space point. No dilation here. */
static void ewa_cov2d(const orc_camera* cam, const double pc[3], const float* scale,
                      const float* quat, double cov2d[3]) {
  double Rq[9];
  quat_to_rotation(quat, Rq);
  double M[9]; /* Rq * diag(s) */
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) M[3 * r + c] = Rq[3 * r + c] * (double)scale[c];
  double S3[9]; /* M M^T */
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += M[3 * r + k] * M[3 * c + k];
      S3[3 * r + c] = acc;
    }
  const double z = pc[2];
  const double limx = 1.3 * (0.5 * cam->width / cam->fx);
  const double limy = 1.3 * (0.5 * cam->height / cam->fy);
  double xz = pc[0] / z, yz = pc[1] / z;
  xz = xz < -limx ? -limx : (xz > limx ? limx : xz);
  yz = yz < -limy ? -limy : (yz > limy ? limy : yz);
  const double tx = xz * z, ty = yz * z;
  double J[6] = {cam->fx / z, 0.0, -cam->fx * tx / (z * z),
                 0.0, cam->fy / z, -cam->fy * ty / (z * z)};
  double T[6]; /* J W */
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += J[3 * r + k] * cam->R[3 * k + c];
      T[3 * r + c] = acc;
    }
  double TS[6]; /* T Sigma */
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += T[3 * r + k] * S3[3 * k + c];
      TS[3 * r + c] = acc;
    }
  double C2[4]; /* T Sigma T^T */
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += TS[3 * r + k] * T[3 * c + k];
      C2[2 * r + c] = acc;
    }
  cov2d[0] = C2[0];
  cov2d[1] = 0.5 * (C2[1] + C2[2]);
  cov2d[2] = C2[3];
}

void orc_project_cov(const float* mean, const float* scale, const float* quat,
                     const orc_camera* cam, double cov2d[3]) {
  double pc[3];
  to_camera(cam, mean, pc);
  ewa_cov2d(cam, pc, scale, quat, cov2d);
}

static int64_t floor_div16(int64_t v) { return v >= 0 ? v / ORC_TILE : -((-v + ORC_TILE - 1) / ORC_TILE); }

int32_t orc_tile_rect(double mx, double my, int32_t r, int32_t width, int32_t height,
                      int32_t rect[4]) {
  /* pixel i is inside [m - r, m + r] iff ceil(m) - r <= i <= floor(m) + r (r is an integer) */
  const int64_t bx0 = (int64_t)ceil(mx) - r, bx1 = (int64_t)floor(mx) + r;
  const int64_t by0 = (int64_t)ceil(my) - r, by1 = (int64_t)floor(my) + r;
  const int64_t px0 = bx0 > 0 ? bx0 : 0, px1 = bx1 < width - 1 ? bx1 : width - 1;
  const int64_t py0 = by0 > 0 ? by0 : 0, py1 = by1 < height - 1 ? by1 : height - 1;
  if (px0 > px1 || py0 > py1) {
    rect[0] = rect[1] = rect[2] = rect[3] = 0;
    return 0;
  }
  rect[0] = (int32_t)floor_div16(px0);
  rect[1] = (int32_t)floor_div16(py0);
  rect[2] = (int32_t)floor_div16(px1) + 1;
  rect[3] = (int32_t)floor_div16(py1) + 1;
  return 1;
}

void orc_preprocess(int64_t n, int32_t sh_degree, const float* means, const float* scales,
                    const float* quats, const float* opacities, const float* sh,
                    const orc_camera* cam, double* mean2d, double* conic, double* opacity,
                    double* rgb, double* depth, int32_t* radius, int32_t* rect) {
  const int nc = (sh_degree + 1) * (sh_degree + 1);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    mean2d[2 * i] = mean2d[2 * i + 1] = 0.0;
    conic[3 * i] = conic[3 * i + 1] = conic[3 * i + 2] = 0.0;
    opacity[i] = 0.0;
    rgb[3 * i] = rgb[3 * i + 1] = rgb[3 * i + 2] = 0.0;
    depth[i] = 0.0;
    radius[i] = 0;
    rect[4 * i] = rect[4 * i + 1] = rect[4 * i + 2] = rect[4 * i + 3] = 0;

    double pc[3];
    to_camera(cam, means + 3 * i, pc);
    if (!(pc[2] > cam->near_z)) continue; /* frustum culling (near plane) */

    double cov[3];
    ewa_cov2d(cam, pc, scales + 3 * i, quats + 4 * i, cov);
    cov[0] += 0.3;
    cov[2] += 0.3;
    const double det = cov[0] * cov[2] - cov[1] * cov[1];
    if (!(det > 0.0)) continue;
    const double ca = cov[2] / det, cb = -cov[1] / det, cc = cov[0] / det;

    const double mx = cam->fx * pc[0] / pc[2] + cam->cx;
    const double my = cam->fy * pc[1] / pc[2] + cam->cy;

    const double mid = 0.5 * (cov[0] + cov[2]);
    double disc = mid * mid - det;
    if (disc < 0.1) disc = 0.1;
    const double l1 = mid + sqrt(disc), l2 = mid - sqrt(disc);
    const int32_t r = (int32_t)ceil(3.0 * sqrt(l1 > l2 ? l1 : l2));

    int32_t rc[4];
    if (!orc_tile_rect(mx, my, r, cam->width, cam->height, rc)) continue;

    /* colour: SH evaluated along the normalized view direction, + 0.5, clamped at 0 */
    double dir[3] = {(double)means[3 * i] - cam->cam_pos[0], (double)means[3 * i + 1] - cam->cam_pos[1],
                     (double)means[3 * i + 2] - cam->cam_pos[2]};
    const double dn = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    dir[0] /= dn; dir[1] /= dn; dir[2] /= dn;
    double Y[16];
    orc_sh_basis(dir, Y);
    for (int ch = 0; ch < 3; ++ch) {
      double acc = 0.0;
      for (int k = 0; k < nc; ++k) acc += (double)sh[((int64_t)i * nc + k) * 3 + ch] * Y[k];
      acc += 0.5;
      rgb[3 * i + ch] = acc > 0.0 ? acc : 0.0;
    }

    mean2d[2 * i] = mx;
    mean2d[2 * i + 1] = my;
    conic[3 * i] = ca;
    conic[3 * i + 1] = cb;
    conic[3 * i + 2] = cc;
    opacity[i] = (double)opacities[i];
    depth[i] = pc[2];
    radius[i] = r;
    memcpy(rect + 4 * i, rc, sizeof rc);
  }
}

/* --------------------------------------------------------------------------------------------
 * Group-level entries (Section 4.4.2; Algorithm 1). */
static void group_grid(int32_t width, int32_t height, int32_t gw, int32_t gh, int32_t* TX,
                       int32_t* TY, int32_t* GX, int32_t* GY) {
  *TX = (width + ORC_TILE - 1) / ORC_TILE;
  *TY = (height + ORC_TILE - 1) / ORC_TILE;
  *GX = (*TX + gw - 1) / gw;
  *GY = (*TY + gh - 1) / gh;
}

/* Tile membership. A (splat, tile) pair can matter only where alpha = o e^power >= 1/255, i.e.
 * inside the ellipse Q(d) = a dx^2 + 2 b dx dy + c dy^2 <= 2 ln(255 o). The rule widens that level
 * to R = 2 (ln 255 + L(o) + 0.05), with L(o) >= ln(o) read off the float's exponent and mantissa
 * (L = k ln 2 + ln 2 / 2 if the mantissa is below sqrt 2, else (k + 1) ln 2), and widens every tile's
 * pixel-centre box [16 tx, 16 tx + 15] x [16 ty, 16 ty + 15] by 1/16 px. The ellipse is convex, so
 * in the band of tile row ty the tiles it meets are one run [lo, hi]: from the x-extent of the
 * ellipse inside the band, which is attained at the band's point nearest to the ellipse's
 * rightmost (leftmost) point, dy = -(b/c) Xmax (+(b/c) Xmax), Xmax = sqrt(R c / det).
 * Every value is a float and every operation rounds to float on its own (no contraction; the one
 * fmaf is Kahan's determinant): the CUDA path takes the same decisions bit for bit. */
#define ORC_MEMBER_EPS 0.0625f
#define ORC_MEMBER_MARGIN 0.05f

typedef struct {
  float mx, my, ia, b, det, aR, Xmax, Ymax, bc;
  int all;  /* degenerate conic: keep every tile of the range */
  int none; /* o < 1/255: no tile */
} orc_member;

static void member_setup(float mx, float my, float a, float b, float c, float o, orc_member* g) {
  memset(g, 0, sizeof *g);
  g->mx = mx;
  g->my = my;
  g->b = b;
  const float w = b * b;
  const float e = fmaf(-b, b, w); /* w - b b exactly */
  const float det = fmaf(a, c, -w) + e;
  if (!(a > 0.0f) || !(c > 0.0f) || !(det > 0.0f)) {
    g->all = 1;
    return;
  }
  uint32_t bits;
  memcpy(&bits, &o, sizeof bits);
  const int32_t ex = (int32_t)((bits >> 23) & 0xFFu);
  const uint32_t man = bits & 0x7FFFFFu;
  /* L(o) = halves * (ln 2) / 2; 0x3504F3 is the mantissa of the largest float below sqrt 2 */
  const int32_t halves = ex == 0 ? -250 : 2 * (ex - 127) + (man <= 0x3504F3u ? 1 : 2);
  const float L = (float)halves * 0.3465736f;
  float t = 5.5412636f + L; /* ln 255 */
  t = t + ORC_MEMBER_MARGIN;
  const float R = 2.0f * t;
  if (!(R > 0.0f)) {
    g->none = 1;
    return;
  }
  const float aR = a * R;
  const float cR = c * R;
  g->aR = aR;
  g->det = det;
  g->Ymax = sqrtf(aR / det);
  g->Xmax = sqrtf(cR / det);
  g->bc = b / c;
  g->ia = 1.0f / a;
}

static float clampf(float v, float lo, float hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* The tiles [*lo, *hi] of tile row ty the ellipse meets (*lo > *hi: none). */
static void member_row(const orc_member* g, int32_t ty, int32_t* lo, int32_t* hi) {
  const float y0 = (float)(16 * ty) - ORC_MEMBER_EPS;
  const float y1 = (float)(16 * ty + 15) + ORC_MEMBER_EPS;
  const float dy0 = y0 - g->my;
  const float dy1 = y1 - g->my;
  const float nY = -g->Ymax;
  const float lb = dy0 > nY ? dy0 : nY;
  const float ub = dy1 < g->Ymax ? dy1 : g->Ymax;
  if (!(lb <= ub)) {
    *lo = 1;
    *hi = 0;
    return;
  }
  const float sx = g->bc * g->Xmax;
  const float yh = clampf(-sx, lb, ub);
  const float yl = clampf(sx, lb, ub);
  const float dh = g->det * yh;
  const float dl = g->det * yl;
  const float qh = g->aR - dh * yh;
  const float ql = g->aR - dl * yl;
  const float sh = sqrtf(qh > 0.0f ? qh : 0.0f);
  const float sl = sqrtf(ql > 0.0f ? ql : 0.0f);
  const float bh = g->b * yh;
  const float bl = g->b * yl;
  const float xh = (sh - bh) * g->ia;
  const float xl = (-sl - bl) * g->ia;
  const float xmax = g->mx + xh;
  const float xmin = g->mx + xl;
  const float fh = clampf((xmax + ORC_MEMBER_EPS) * 0.0625f, -1e6f, 1e6f);
  const float fl = clampf((xmin - (15.0f + ORC_MEMBER_EPS)) * 0.0625f, -1e6f, 1e6f);
  *hi = (int32_t)floorf(fh);
  *lo = (int32_t)ceilf(fl);
}

/* Mask of the member tiles of group (gx, gy) that are in the tile range `rc` and, with membership,
 * meet the splat's ellipse. */
static uint32_t group_mask(const orc_member* g, const int32_t rc[4], int32_t gx, int32_t gy,
                           int32_t gw, int32_t gh) {
  uint32_t mask = 0;
  for (int32_t ty = gy * gh; ty < (gy + 1) * gh; ++ty) {
    if (ty < rc[1] || ty >= rc[3]) continue;
    int32_t lo = rc[0], hi = rc[2] - 1;
    if (g && !g->all) {
      if (g->none) continue;
      int32_t rl, rh;
      member_row(g, ty, &rl, &rh);
      if (rl > lo) lo = rl;
      if (rh < hi) hi = rh;
    }
    for (int32_t tx = gx * gw; tx < (gx + 1) * gw; ++tx)
      if (tx >= lo && tx <= hi) mask |= 1u << ((ty - gy * gh) * gw + (tx - gx * gw));
  }
  return mask;
}

struct orc_entry_s;

/* Counts or fills (when ent != NULL) the entries of every visible splat: one per group of its tile
 * range whose mask (with membership when conic != NULL) is not empty. */
static int64_t enumerate_entries(int64_t n, const double* mean2d, const int32_t* radius,
                                 const double* depth, const double* conic, const double* opacity,
                                 int32_t width, int32_t height, int32_t gw, int32_t gh, int32_t GX,
                                 struct orc_entry_s* ent);

int64_t orc_bin_count(int64_t n, const double* mean2d, const int32_t* radius, const double* conic,
                      const double* opacity, int32_t width, int32_t height, int32_t gw, int32_t gh) {
  const int32_t GX = ((width + ORC_TILE - 1) / ORC_TILE + gw - 1) / gw;
  return enumerate_entries(n, mean2d, radius, NULL, conic, opacity, width, height, gw, gh, GX, NULL);
}

typedef struct orc_entry_s {
  uint64_t key;
  uint32_t val;
  uint16_t mask;
} orc_entry;

static int entry_cmp(const void* pa, const void* pb) {
  const orc_entry* a = (const orc_entry*)pa;
  const orc_entry* b = (const orc_entry*)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  if (a->val != b->val) return a->val < b->val ? -1 : 1;
  return 0;
}

static uint32_t float_bits(double v) {
  const float f = (float)v;
  uint32_t u;
  memcpy(&u, &f, sizeof u);
  return u;
}

static int64_t enumerate_entries(int64_t n, const double* mean2d, const int32_t* radius,
                                 const double* depth, const double* conic, const double* opacity,
                                 int32_t width, int32_t height, int32_t gw, int32_t gh, int32_t GX,
                                 orc_entry* ent) {
  int64_t e = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (radius[i] <= 0) continue;
    int32_t rc[4];
    if (!orc_tile_rect(mean2d[2 * i], mean2d[2 * i + 1], radius[i], width, height, rc)) continue;
    orc_member m;
    if (conic)
      member_setup((float)mean2d[2 * i], (float)mean2d[2 * i + 1], (float)conic[3 * i],
                   (float)conic[3 * i + 1], (float)conic[3 * i + 2], (float)opacity[i], &m);
    const uint32_t dbits = ent ? float_bits(depth[i]) : 0u;
    for (int32_t gy = rc[1] / gh; gy <= (rc[3] - 1) / gh; ++gy)
      for (int32_t gx = rc[0] / gw; gx <= (rc[2] - 1) / gw; ++gx) {
        const uint32_t mask = group_mask(conic ? &m : NULL, rc, gx, gy, gw, gh);
        if (!mask) continue;
        if (ent) {
          ent[e].key = ((uint64_t)(uint32_t)(gy * GX + gx) << 32) | dbits;
          ent[e].val = (uint32_t)i;
          ent[e].mask = (uint16_t)mask;
        }
        ++e;
      }
  }
  return e;
}

void orc_bin(int64_t n, const double* mean2d, const int32_t* radius, const double* depth,
             const double* conic, const double* opacity, int32_t width, int32_t height, int32_t gw,
             int32_t gh, uint64_t* keys, uint32_t* vals, uint16_t* masks, uint32_t* ranges) {
  int32_t TX, TY, GX, GY;
  group_grid(width, height, gw, gh, &TX, &TY, &GX, &GY);
  const int64_t E = enumerate_entries(n, mean2d, radius, depth, conic, opacity, width, height, gw,
                                      gh, GX, NULL);
  orc_entry* ent = (orc_entry*)malloc((size_t)(E > 0 ? E : 1) * sizeof(orc_entry));
  enumerate_entries(n, mean2d, radius, depth, conic, opacity, width, height, gw, gh, GX, ent);
  qsort(ent, (size_t)E, sizeof(orc_entry), entry_cmp);
  for (int64_t g = 0; g < (int64_t)GX * GY; ++g) ranges[2 * g] = ranges[2 * g + 1] = 0;
  for (int64_t k = 0; k < E; ++k) {
    keys[k] = ent[k].key;
    vals[k] = ent[k].val;
    masks[k] = ent[k].mask;
    const uint32_t g = (uint32_t)(ent[k].key >> 32);
    if (k == 0 || (uint32_t)(ent[k - 1].key >> 32) != g) ranges[2 * g] = (uint32_t)k;
    ranges[2 * g + 1] = (uint32_t)(k + 1);
  }
  free(ent);
}

/* --------------------------------------------------------------------------------------------
 * Front-to-back blending (Section 2). */
static double dmin(double a, double b) { return a < b ? a : b; }

void orc_blend(int32_t width, int32_t height, int32_t gw, int32_t gh, const double* mean2d,
               const double* conic, const double* opacity, const double* rgb, const uint32_t* vals,
               const uint16_t* masks, const uint32_t* ranges, const double bg[3],
               const int32_t* pix, int64_t npix, double* out_rgb, double* out_T,
               int32_t* n_contrib, double* margin, int64_t* counters) {
  int32_t TX, TY, GX, GY;
  group_grid(width, height, gw, gh, &TX, &TY, &GX, &GY);
  const int64_t count = pix ? npix : (int64_t)width * height;
  int64_t evaluated = 0, guard = 0, passing = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : evaluated, guard, passing)
  for (int64_t p = 0; p < count; ++p) {
    const int32_t x = pix ? pix[2 * p] : (int32_t)(p % width);
    const int32_t y = pix ? pix[2 * p + 1] : (int32_t)(p / width);
    const int32_t tx = x / ORC_TILE, ty = y / ORC_TILE;
    const int32_t gx = tx / gw, gy = ty / gh;
    const int64_t gid = (int64_t)gy * GX + gx;
    const int bit = (ty - gy * gh) * gw + (tx - gx * gw);
    double T = 1.0, C[3] = {0.0, 0.0, 0.0}, mg = 1.0;
    int32_t last = 0;
    const uint32_t start = ranges[2 * gid], end = ranges[2 * gid + 1];
    for (uint32_t k = start; k < end; ++k) {
      if (!((masks[k] >> bit) & 1u)) continue; /* entry does not overlap this tile */
      const uint32_t i = vals[k];
      ++evaluated;
      const double dx = (double)x - mean2d[2 * i], dy = (double)y - mean2d[2 * i + 1]; /* Eq. power_d */
      const double a = conic[3 * i], b = conic[3 * i + 1], c = conic[3 * i + 2];
      const double power = -0.5 * a * dx * dx - b * dx * dy - 0.5 * c * dy * dy; /* Eq. tensorgs_power_scalar */
      if (power > 0.0) {
        ++guard;
        continue;
      }
      const double oe = opacity[i] * exp(power);
      const double alpha = dmin(0.99, oe);
      mg = dmin(mg, fabs(oe * 255.0 - 1.0));
      if (alpha < 1.0 / 255.0) continue; /* prune a negligible contribution */
      ++passing;
      const double Tn = T * (1.0 - alpha);
      mg = dmin(mg, fabs(Tn / 1e-4 - 1.0));
      if (Tn < 1e-4) break; /* early termination: this entry is not blended */
      for (int ch = 0; ch < 3; ++ch) C[ch] += alpha * T * rgb[3 * i + ch];
      T = Tn;
      last = (int32_t)(k - start + 1);
    }
    for (int ch = 0; ch < 3; ++ch) out_rgb[3 * p + ch] = C[ch] + T * bg[ch];
    out_T[p] = T;
    n_contrib[p] = last;
    margin[p] = mg;
  }
  counters[0] += evaluated;
  counters[1] += guard;
  counters[2] += passing;
}

/* --------------------------------------------------------------------------------------------
 * Backward of the blend. For pixel p with blended entries i = 1..m (alpha_i, T_i), colour
 * C = sum_i alpha_i T_i c_i + T_final bg. With B_i = (sum_{j>i} alpha_j T_j c_j + T_final bg) / T_{i+1}:
 *   dC/dc_i = alpha_i T_i,  dC/dalpha_i = T_i (c_i - B_i),  B_{i-1} = alpha_i c_i + (1 - alpha_i) B_i,
 * alpha = o e^power unless clamped at 0.99 (then dalpha = 0): dalpha/do = e^power, dalpha/dpower = alpha,
 * dpower/d(a, b, c) = (-dx^2/2, -dx dy, -dy^2/2), dpower/dmu = (a dx + b dy, b dx + c dy).
 * The forward replay stores each blended entry; no division is needed. Serial over pixels so the
 * accumulation order is fixed. */
typedef struct {
  uint32_t i;
  double alpha, T, ep, dx, dy;
  int clamped;
} orc_step;

void orc_blend_backward(int32_t width, int32_t height, int32_t gw, int32_t gh,
                        int64_t n, const double* mean2d, const double* conic,
                        const double* opacity, const double* rgb, const uint32_t* vals,
                        const uint16_t* masks, const uint32_t* ranges, const double bg[3],
                        const int32_t* pix, int64_t npix, const double* grad_rgb,
                        double* g_mean2d, double* g_conic, double* g_opacity, double* g_rgb) {
  int32_t TX, TY, GX, GY;
  group_grid(width, height, gw, gh, &TX, &TY, &GX, &GY);
  memset(g_mean2d, 0, sizeof(double) * 2 * (size_t)n);
  memset(g_conic, 0, sizeof(double) * 3 * (size_t)n);
  memset(g_opacity, 0, sizeof(double) * (size_t)n);
  memset(g_rgb, 0, sizeof(double) * 3 * (size_t)n);
  const int64_t count = pix ? npix : (int64_t)width * height;
  size_t cap = 256;
  orc_step* st = (orc_step*)malloc(cap * sizeof(orc_step));
  for (int64_t p = 0; p < count; ++p) {
    const int32_t x = pix ? pix[2 * p] : (int32_t)(p % width);
    const int32_t y = pix ? pix[2 * p + 1] : (int32_t)(p / width);
    const int32_t tx = x / ORC_TILE, ty = y / ORC_TILE;
    const int32_t gx = tx / gw, gy = ty / gh;
    const int64_t gid = (int64_t)gy * GX + gx;
    const int bit = (ty - gy * gh) * gw + (tx - gx * gw);
    const double* G = grad_rgb + 3 * p;
    /* forward replay, identical decisions to orc_blend */
    size_t m = 0;
    double T = 1.0;
    for (uint32_t k = ranges[2 * gid]; k < ranges[2 * gid + 1]; ++k) {
      if (!((masks[k] >> bit) & 1u)) continue;
      const uint32_t i = vals[k];
      const double dx = (double)x - mean2d[2 * i], dy = (double)y - mean2d[2 * i + 1];
      const double a = conic[3 * i], b = conic[3 * i + 1], c = conic[3 * i + 2];
      const double power = -0.5 * a * dx * dx - b * dx * dy - 0.5 * c * dy * dy;
      if (power > 0.0) continue;
      const double ep = exp(power);
      const double oe = opacity[i] * ep;
      const double alpha = dmin(0.99, oe);
      if (alpha < 1.0 / 255.0) continue;
      const double Tn = T * (1.0 - alpha);
      if (Tn < 1e-4) break;
      if (m == cap) {
        cap *= 2;
        st = (orc_step*)realloc(st, cap * sizeof(orc_step));
      }
      st[m].i = i; st[m].alpha = alpha; st[m].T = T; st[m].ep = ep;
      st[m].dx = dx; st[m].dy = dy; st[m].clamped = oe > 0.99;
      ++m;
      T = Tn;
    }
    /* reverse pass */
    double B[3] = {bg[0], bg[1], bg[2]};
    for (size_t s = m; s-- > 0;) {
      const uint32_t i = st[s].i;
      const double alpha = st[s].alpha, Ti = st[s].T;
      double dL_dalpha = 0.0;
      for (int ch = 0; ch < 3; ++ch) {
        const double ci = rgb[3 * i + ch];
        g_rgb[3 * i + ch] += alpha * Ti * G[ch];
        dL_dalpha += G[ch] * Ti * (ci - B[ch]);
        B[ch] = alpha * ci + (1.0 - alpha) * B[ch];
      }
      if (st[s].clamped) continue;
      const double dx = st[s].dx, dy = st[s].dy;
      const double a = conic[3 * i], b = conic[3 * i + 1], c = conic[3 * i + 2];
      const double dL_dpower = dL_dalpha * alpha;
      g_opacity[i] += dL_dalpha * st[s].ep;
      g_conic[3 * i] += dL_dpower * (-0.5 * dx * dx);
      g_conic[3 * i + 1] += dL_dpower * (-dx * dy);
      g_conic[3 * i + 2] += dL_dpower * (-0.5 * dy * dy);
      g_mean2d[2 * i] += dL_dpower * (a * dx + b * dy);
      g_mean2d[2 * i + 1] += dL_dpower * (b * dx + c * dy);
    }
  }
  free(st);
}
