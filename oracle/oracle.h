/* FP64 CPU oracle of the tile-based 3D Gaussian Splatting rasterizer with cross-tile grouping.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg may load this library. The rendering library never links, loads or calls it, and the two
 * share no code.
 *
 * Every function follows the definitions of "Accelerating 3D Gaussian Splatting using Tensor
 * Cores" (TensorGS), Section 2 and Section 4, in plain double precision with no blocking, fusion or
 * reordering beyond what the definitions state. Where the paper is silent the header of oracle.c
 * states the reading taken.
 */
#ifndef TGS_ORACLE_H
#define TGS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_TILE 16

typedef struct {
  int32_t width, height;
  double fx, fy, cx, cy;
  double R[9];       /* world -> camera rotation, row-major */
  double t[3];       /* world -> camera translation */
  double cam_pos[3]; /* camera centre in world coordinates */
  double near_z;     /* camera-space z <= near_z is culled */
} orc_camera;

/* Real spherical-harmonic basis up to degree 3 at unit direction d (Section 2: view-dependent
 * colour from SH coefficients). out[l*l + m + l] for m = -l..l. */
void orc_sh_basis(const double d[3], double out[16]);

/* Frustum culling + feature computation (Section 2, Algorithm 1 lines "Frustum-cull" and
 * "Compute screen-space attributes"). Outputs per splat; radius[i] == 0 marks a culled splat
 * (then the other outputs of i are zero). rect = tile range [tx0, tx1) x [ty0, ty1). */
void orc_preprocess(int64_t n, int32_t sh_degree, const float* means, const float* scales,
                    const float* quats, const float* opacities, const float* sh,
                    const orc_camera* cam, double* mean2d, double* conic, double* opacity,
                    double* rgb, double* depth, int32_t* radius, int32_t* rect);

/* Projected covariance of one splat before dilation (EWA, Section 2), for tests. */
void orc_project_cov(const float* mean, const float* scale, const float* quat,
                     const orc_camera* cam, double cov2d[3]);

/* Tile range of the AABB [mu - r, mu + r]^2 against the pixel grid: the tiles that hold at least
 * one image pixel inside it. Returns 0 if empty. */
int32_t orc_tile_rect(double mx, double my, int32_t r, int32_t width, int32_t height,
                      int32_t rect[4]);

/* Number of group-level entries (Section 4.4.2: one entry per overlapped tile group whose mask is
 * not empty). conic [n,3] and opacity [n] (FP32 values) switch on the tile-membership test (see
 * oracle.c); NULL keeps every tile of the AABB's range. */
int64_t orc_bin_count(int64_t n, const double* mean2d, const int32_t* radius, const double* conic,
                      const double* opacity, int32_t width, int32_t height, int32_t gw, int32_t gh);

/* Group-level entries with tile-membership masks, sorted by (group ID, depth) (Section 4.4.2,
 * Algorithm 1). keys = (gid << 32) | bits(float(depth)); ties by splat index. ranges[2g], ranges[2g+1]
 * = [start, end) of group g. conic / opacity as in orc_bin_count. */
void orc_bin(int64_t n, const double* mean2d, const int32_t* radius, const double* depth,
             const double* conic, const double* opacity, int32_t width, int32_t height, int32_t gw,
             int32_t gh, uint64_t* keys, uint32_t* vals, uint16_t* masks, uint32_t* ranges);

/* Front-to-back blending of every pixel (Section 2 Eqs. power_d, power, alpha, blend; pruning and
 * early termination). If pix != NULL only the npix listed pixels (x, y pairs) are computed and the
 * outputs are indexed by list position; otherwise all pixels, row-major.
 * margin = smallest relative distance of any threshold decision from its threshold (1 = none).
 * counters[0] += evaluated (pixel, entry) pairs; counters[1] += power > 0 guard firings;
 * counters[2] += evaluated pairs with alpha >= 1/255 (those that need the exponential). */
void orc_blend(int32_t width, int32_t height, int32_t gw, int32_t gh, const double* mean2d,
               const double* conic, const double* opacity, const double* rgb, const uint32_t* vals,
               const uint16_t* masks, const uint32_t* ranges, const double bg[3],
               const int32_t* pix, int64_t npix, double* out_rgb, double* out_T,
               int32_t* n_contrib, double* margin, int64_t* counters);

/* Gradient of L = sum(out_rgb * grad_rgb) with respect to mean2d, conic (a, b, c), opacity and
 * rgb of every splat, by the analytic chain rule through the blend in reverse order. Outputs are
 * overwritten. Pixels listed as in orc_blend (NULL = all). */
void orc_blend_backward(int32_t width, int32_t height, int32_t gw, int32_t gh,
                        int64_t n, const double* mean2d, const double* conic,
                        const double* opacity, const double* rgb, const uint32_t* vals,
                        const uint16_t* masks, const uint32_t* ranges, const double bg[3],
                        const int32_t* pix, int64_t npix, const double* grad_rgb,
                        double* g_mean2d, double* g_conic, double* g_opacity, double* g_rgb);

int32_t orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
