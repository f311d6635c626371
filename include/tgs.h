/* tgs.h -- C ABI of a GB300 (sm_103a) tensor-core 3D Gaussian Splatting rasterizer.
 *
 * The operations follow "Accelerating 3D Gaussian Splatting using Tensor Cores" (TensorGS):
 *   tgs_preprocess          Section 2 "Frustum culling" and "Feature computation"; Algorithm 1,
 *                           "Frustum-cull visible Gaussians" and "Compute screen-space attributes".
 *   tgs_bin_sort            Section 2 "Gaussian sorting" with the grouped list of Section 4.4.2
 *                           ("Constructing the grouped Gaussian list"); Algorithm 1, the per-group
 *                           entry generation with tile-membership masks and the sort by
 *                           (group ID, depth).
 *   tgs_rasterize           Section 2 "Rasterization" (Eqs. power_d, power, alpha, blend, pruning
 *                           and early termination), tensorized as in Section 4.2 and grouped as in
 *                           Section 4.4.2; Algorithm 1, the per-group CTA loop.
 *   tgs_rasterize_backward  Gradients of the blend of Section 2 (the paper trains Gaussian models,
 *                           Section 3.2.1, but prints no backward; the chain rule of the forward).
 *   tgs_serve_*             A multi-scene rendering service built on the three calls above (the
 *                           paper motivates frame-latency budgets in Section 1; it has no server).
 *
 * Conventions shared by every call:
 *   - Every function returns a tgs_status; TGS_OK is 0. No C++ exception crosses the ABI.
 *   - Argument errors are reported synchronously, before any work is enqueued. Errors of kernels
 *     surface from the CUDA runtime at a later call or stream synchronization.
 *   - Device pointers are caller-owned, contiguous, row-major. Floating point is FP32 unless stated.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). All work is enqueued on it;
 *     no call synchronizes the stream unless its comment says so.
 *   - The library allocates device memory only inside objects it creates (tgs_server). Its
 *     device error word (one int32 per device) is a variable of the library's own device code,
 *     not an allocation. The bin sort takes a caller-provided workspace sized by
 *     tgs_bin_sort_workspace_size.
 *   - The library caches per-device state (the error word's address, the static scratch's
 *     address) for the life of the process: do not use it again after cudaDeviceReset.
 *   - The image is sampled at integer pixel coordinates: pixel (i, j) is at (x, y) = (i, j).
 *     Tiles are 16x16 pixels. A tile group is group_w x group_h tiles (1x1 up to 4x4).
 */
#ifndef TGS_H
#define TGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TGS_ABI_VERSION 3
#define TGS_TILE 16
#define TGS_MAX_GROUP 4

typedef int32_t tgs_status;
#define TGS_OK 0
#define TGS_ERR_INVALID_ARGUMENT 1  /* a pointer, size or option is out of range */
#define TGS_ERR_CUDA 2              /* a CUDA runtime call failed; see tgs_last_error_message */
#define TGS_ERR_CAPACITY 3          /* more bin entries than the caller's capacity */
#define TGS_ERR_UNSUPPORTED_DEVICE 4 /* the current device is not compute capability 10.3 */
#define TGS_ERR_TIMEOUT 5           /* a bounded wait expired (device pipeline or service) */
#define TGS_ERR_BUSY 6              /* the service cannot admit the request now */
#define TGS_ERR_NOT_FOUND 7         /* unknown scene id or ticket */

/* Precision of the rasterizer's exponent evaluation (the "power" of Eq. power). */
#define TGS_PRECISION_FP32 0    /* scalar FP32 on the CUDA cores (the plain tile rasterizer) */
#define TGS_PRECISION_FP16_TC 1 /* FP16 x FP16 -> FP32 product on the tensor cores (tcgen05) */
#define TGS_PRECISION_BF16_TC 2 /* BF16 x BF16 -> FP32 product on the tensor cores (tcgen05), the
                                   coefficients split three ways over K = 32 */

typedef struct {
  int64_t n;              /* number of Gaussians */
  int32_t sh_degree;      /* 0..3 */
  const float* means;     /* [n,3] world-space means */
  const float* scales;    /* [n,3] linear standard deviations along the local axes */
  const float* quats;     /* [n,4] rotation quaternions (w, x, y, z); normalized inside */
  const float* opacities; /* [n]   opacity in (0, 1) */
  const float* sh;        /* [n,(sh_degree+1)^2,3] SH coefficients, index l*l + m + l */
} tgs_scene;

typedef struct {
  int32_t width, height;  /* image size in pixels, 1..16384 each */
  float fx, fy, cx, cy;   /* pinhole intrinsics: u = fx x/z + cx, v = fy y/z + cy */
  float R[9];             /* world -> camera rotation, row-major (camera x right, y down, z fwd) */
  float t[3];             /* world -> camera translation: p_cam = R p_world + t */
  float cam_pos[3];       /* camera centre in world coordinates (SH view direction origin) */
  float near_z;           /* Gaussians with camera-space z <= near_z are culled */
} tgs_camera;

/* Flags of tgs_tiling. */
#define TGS_BIN_RANGE_ONLY 1 /* keep every tile of a Gaussian's AABB tile range (no membership
                                test; for measuring the test, the image is the same) */

typedef struct {
  int32_t group_w, group_h; /* tiles per group along x and y, each 1..TGS_MAX_GROUP */
  int32_t flags;            /* TGS_BIN_*; 0 = tile membership on */
} tgs_tiling;

/* Projected Gaussians: caller-allocated device arrays of length n (written by tgs_preprocess,
 * read by tgs_bin_sort / tgs_rasterize / tgs_rasterize_backward). */
typedef struct {
  float* mean2d;        /* [n,2] projected mean mu' in pixels */
  float* conic_opacity; /* [n,4] (a, b, c, o): inverse projected covariance [[a,b],[b,c]], opacity */
  float* rgb;           /* [n,3] SH colour, clamped at 0 */
  float* depth;         /* [n]   camera-space z */
  int32_t* radius;      /* [n]   ceil(3 sqrt(lambda_max)) in pixels; 0 = culled (then the other
                           arrays of that Gaussian are not written) */
  int32_t* rect;        /* [n,4] overlapped tile range (tx0, ty0, tx1, ty1), max exclusive */
} tgs_projected;

/* Sorted group-level entries (Section 4.4.2). Arrays are caller-allocated device memory. */
typedef struct {
  int64_t capacity;     /* number of entries keys/vals/masks can hold (< 2^30) */
  uint64_t* keys;       /* [capacity] (group id << 32) | bits(float depth), ascending; may be NULL */
  uint32_t* vals;       /* [capacity] Gaussian index of each entry */
  uint16_t* masks;      /* [capacity] tile-membership bits, bit (ty%gh)*gw + (tx%gw) */
  uint32_t* ranges;     /* [num_groups,2] [start, end) per group, row-major groups; (0,0) if empty */
  int64_t* num_entries; /* device scalar: entries needed by this frame (may exceed capacity) */
} tgs_bins;

/* Flags of tgs_raster_opts. */
#define TGS_RASTER_NO_CULL 1 /* FP16_TC: do not skip (Gaussian, tile) pairs whose exponent cannot
                                reach log2(1/255) anywhere in the tile (the skip never changes the
                                image; this flag exists to measure it) */

typedef struct {
  int32_t precision;    /* TGS_PRECISION_* */
  int32_t flags;        /* TGS_RASTER_* */
  float bg[3];          /* background colour added as T_final * bg */
  int64_t* counters;    /* optional device [3] int64, accumulated: [0] (pixel, entry) pairs
                           evaluated before termination (mask bit set; FP16_TC does not count the
                           pairs of a tile it skipped as provably below 1/255), [1] of those, the
                           pairs with alpha >= 1/255 (each needs one exp), [2] (pixel, list slot)
                           steps the kernel issued, terminated pixels, other tiles' entries and
                           padding included (its work granularity); NULL = not counted */
} tgs_raster_opts;

/* ---------------------------------------------------------------------------------------------- */

const char* tgs_status_string(tgs_status s);
/* Last error message of the calling host thread ("" if none). Valid until the next call. */
const char* tgs_last_error_message(void);
int32_t tgs_abi_version(void);
/* TGS_OK if `device` is a compute capability 10.3 GPU this library was built for. */
tgs_status tgs_check_device(int32_t device);

/* Preprocess (Section 2: frustum culling, feature computation; Section 4.2.1: conic).
 * Per Gaussian: camera-space mean; cull if z <= near_z; EWA projection of the 3D covariance with the
 * Jacobian taken at x/z, y/z clamped to +-1.3 tan(half FOV); 2D covariance + 0.3 I; conic = its
 * inverse (near-degenerate covariances, det < 2^-5 Sxx Syy, are recomputed in FP64); radius =
 * ceil(3 sqrt(lambda_max)); tile range of the AABB [mu'-r, mu'+r]^2 (tiles holding an image pixel
 * inside it; empty -> culled); SH colour + 0.5 clamped at 0. A culled Gaussian gets radius 0 and
 * its other outputs are left unwritten (no call reads them).
 * Errors: INVALID_ARGUMENT for NULL pointers with n > 0, n < 0, sh_degree outside 0..3, bad camera. */
tgs_status tgs_preprocess(const tgs_scene* scene, const tgs_camera* cam, tgs_projected* out,
                          void* stream);

/* Workspace bytes tgs_bin_sort needs for n Gaussians, `capacity` entries and the image/tiling
 * (n < 2^30 and capacity < 2^30, else TGS_ERR_INVALID_ARGUMENT). */
tgs_status tgs_bin_sort_workspace_size(int64_t n, int64_t capacity, int32_t width, int32_t height,
                                       const tgs_tiling* tiling, size_t* bytes);

/* Bin and sort (Section 4.4.2; Algorithm 1): one entry per (Gaussian, tile group) whose mask of
 * member tiles is not empty, sorted ascending by (group id, float depth, Gaussian index) -- the
 * 64-bit key (gid << 32) | depth bits with ties by index. A tile of the Gaussian's AABB tile range
 * is a member unless the Gaussian provably cannot reach alpha >= 1/255 at any of its pixels (beyond
 * the paper, whose Section 6 cites tighter footprints; the rasterized image is the same; turned off
 * by TGS_BIN_RANGE_ONLY): the Gaussian's ellipse at the level o e^power = e^-0.05 / 255, with o
 * bounded from above by a half power of two, must meet the tile's pixel-centre box widened by 1/16
 * px, tested in FP32 with a fixed operation order. The mask bit of tile (tx, ty) is
 * (ty % gh) * gw + (tx % gw). Fills keys (if non-NULL), vals, masks, ranges and *num_entries (the
 * frame's entry count). Reads proj->rect, depth, radius and, for the membership test, mean2d and
 * conic_opacity. If the frame needs more than `capacity` entries, nothing is emitted, every range
 * is (0, 0) and *num_entries holds the needed count. If num_entries_host != NULL the call copies
 * the count to it, synchronizes `stream` and returns TGS_ERR_CAPACITY on overflow; otherwise it is
 * fully asynchronous. `workspace` is device memory of at least tgs_bin_sort_workspace_size bytes,
 * 256-byte aligned. The radix passes and prefixes wait on earlier tiles (decoupled look-back); a
 * wait that outlasts the limit of tgs_set_lookback_limit records TGS_ERR_TIMEOUT in the device
 * error word (tgs_last_device_error) and the call ends with empty bins (every range (0, 0),
 * *num_entries 0), which rasterize to the background; with num_entries_host the call then returns
 * TGS_ERR_TIMEOUT. */
tgs_status tgs_bin_sort(const tgs_projected* proj, int64_t n, int32_t width, int32_t height,
                        const tgs_tiling* tiling, void* workspace, size_t workspace_bytes,
                        tgs_bins* bins, int64_t* num_entries_host, void* stream);

/* Size of the fixed scratch area tgs_bin_sort_static uses (16 MiB). */
#define TGS_BIN_SORT_STATIC_BYTES ((size_t)16 << 20)

/* tgs_bin_sort without a caller workspace and without any device allocation. The paper has no
 * counterpart: this serves callers that cannot allocate device memory while they run (a real-time
 * frame loop or compositor with a memory budget fixed at start-up, or a host application that owns
 * every device allocation). The scratch is a fixed TGS_BIN_SORT_STATIC_BYTES array inside the
 * library, held by every GPU that loads it until the process exits. No call, the first one
 * included, allocates device memory. Same arguments, outputs and errors as tgs_bin_sort, plus
 * TGS_ERR_CAPACITY with *num_entries_host = -1 (if given) and a message when
 * tgs_bin_sort_workspace_size(n, bins->capacity, ...) exceeds TGS_BIN_SORT_STATIC_BYTES (e.g.
 * about 130k Gaussians with 1M entries); the TGS_ERR_CAPACITY of a frame that needs more entries
 * than bins->capacity leaves the needed count (>= 0) there instead. The first call on a device
 * loads the library's device code on that device (CUDA loads modules lazily), which commits the
 * array's memory, and resolves its address (cudaGetSymbolAddress): make that first call at
 * start-up, before any stream capture on that device. All calls share the array; calls that
 * overlap on the GPU (other streams or host threads) race. */
tgs_status tgs_bin_sort_static(const tgs_projected* proj, int64_t n, int32_t width, int32_t height,
                               const tgs_tiling* tiling, tgs_bins* bins, int64_t* num_entries_host,
                               void* stream);

/* Rasterize (Section 2 Eqs. power_d..blend; Section 4.2 tensorization; Section 4.4.2 grouping).
 * One CTA per tile group walks the group's sorted list in chunks; per pixel, in list order,
 * entries whose mask bit for the pixel's tile is set: power = -1/2 d^T conic d with d = x - mu';
 * alpha = min(0.99, o exp(power)); skip if alpha < 1/255; T' = T (1 - alpha); if T' < 1e-4 the
 * pixel stops without blending this entry; else C += alpha T rgb, T = T'.
 * FP16_TC evaluates log2(o) + log2(e) power as a product of pixel features [x^2, xy, y^2, x, y, 1]
 * (relative to the tile centre, exact in FP16) with per-Gaussian coefficients split hi + lo in FP16,
 * padded to K = 16, accumulated in FP32 in tensor memory; exp and blending are FP32. It skips a
 * (Gaussian, tile) pair when the exact maximum of the exponent over the tile's pixels is below
 * log2(1/255) by a margin (unless TGS_RASTER_NO_CULL): such a pair is pruned at every pixel anyway.
 * Outputs (device, caller-allocated): out_rgb [3,H,W] = C + T bg; out_T [H,W] = final T;
 * n_contrib [H,W] = 1-based position in the group list of the last blended entry (0 = none), may be
 * NULL. Errors: INVALID_ARGUMENT for bad sizes/tiling/precision; UNSUPPORTED_DEVICE for FP16_TC on a
 * device other than sm_103; TIMEOUT can be recorded by the device pipeline (read with
 * tgs_last_device_error after synchronizing). */
tgs_status tgs_rasterize(const tgs_projected* proj, int64_t n, const tgs_bins* bins, int32_t width,
                         int32_t height, const tgs_tiling* tiling, const tgs_raster_opts* opts,
                         float* out_rgb, float* out_T, int32_t* n_contrib, void* stream);

/* Batched tensor-core rasterization: several frames -- of different scenes, resolutions and
 * bins -- rendered by ONE persistent launch (Section 4.4.2's per-group CTA loop over the union of
 * the frames' tile groups; the paper renders one frame at a time and has no counterpart). The work
 * items are the (frame, tile group) pairs; a CTA takes the next item from a device counter until
 * none is left. Each frame's pixels are exactly those tgs_rasterize gives for the same inputs.
 * If frames[f].ready != NULL, frame f's items start only once *ready >= ready_value (device int32,
 * e.g. set by the stream that bins the frame): each CTA waits for it at most wait_limit_ns
 * (<= 0: 2 s); on expiry *status (if non-NULL) is set to TGS_ERR_TIMEOUT and the frame's items
 * are skipped, their pixels left unwritten. status (int32 in device or host-mapped memory,
 * optional) is written only on failure: the caller sets it to TGS_OK before the call. done (int32
 * in device or host-mapped memory, optional) is set to done_value once every item of the frame has
 * been rendered or skipped (after a system-scope fence): a host thread polling it knows when the
 * frame's pixels and status are final, before the whole launch ends. Precision FP16_TC or BF16_TC (FP32:
 * TGS_ERR_INVALID_ARGUMENT; use tgs_rasterize); opts->counters must be NULL. `workspace` is
 * TGS_BATCH_WORKSPACE_BYTES of device memory (the work counter; cleared by the call), owned by the
 * caller and not shared by overlapping calls. Errors: INVALID_ARGUMENT for count outside
 * 1..TGS_BATCH_MAX_FRAMES or a bad frame (reported with its index). */
#define TGS_BATCH_MAX_FRAMES 32
#define TGS_BATCH_WORKSPACE_BYTES 256
typedef struct {
  const tgs_projected* proj; /* the frame's projected Gaussians (as for tgs_rasterize) */
  int64_t n;
  const tgs_bins* bins;      /* its bins, built with the batch's tiling */
  int32_t width, height;
  float* out_rgb;            /* device [3,H,W] */
  float* out_T;              /* device [H,W] */
  const int32_t* ready;      /* optional device readiness flag */
  int32_t ready_value;
  int32_t* status;           /* optional status word */
  int32_t* done;             /* optional completion word */
  int32_t done_value;
} tgs_frame;

tgs_status tgs_rasterize_batch(const tgs_frame* frames, int32_t count, const tgs_tiling* tiling,
                               const tgs_raster_opts* opts, int64_t wait_limit_ns, void* workspace,
                               void* stream);

/* Backward of tgs_rasterize for L = sum(out_rgb * grad_rgb): replays each pixel's list backwards
 * from n_contrib, recovering T_i = T_{i+1} / (1 - alpha_i) from the stored final T. Outputs are
 * overwritten (the call zeroes them first): g_mean2d [n,2] (d/d mu' in pixels), g_conic_opacity
 * [n,4] (d/da, d/db, d/dc, d/do), g_rgb [n,3]. Inputs are those of the forward call plus its
 * out_T and n_contrib. FP32 arithmetic: the forward must have been an FP32 call
 * (opts->precision == TGS_PRECISION_FP32, else TGS_ERR_INVALID_ARGUMENT). */
tgs_status tgs_rasterize_backward(const tgs_projected* proj, int64_t n, const tgs_bins* bins,
                                  int32_t width, int32_t height, const tgs_tiling* tiling,
                                  const tgs_raster_opts* opts, const float* out_T,
                                  const int32_t* n_contrib, const float* grad_rgb,
                                  float* g_mean2d, float* g_conic_opacity, float* g_rgb,
                                  void* stream);

/* Number of CUDA kernels this library has launched in this process (all devices, all threads).
 * A diagnostic for counting the kernels of a timed region. */
int64_t tgs_kernel_launch_count(void);

/* Number of memory allocations (device memory, and pinned host memory) this library has made in
 * this process: only tgs_serve_* objects allocate. A diagnostic for callers that must not
 * allocate. */
int64_t tgs_allocation_count(void);

/* Device-side error word of the library on the current device (TGS_OK or TGS_ERR_TIMEOUT), set by
 * a kernel whose bounded wait expired. Synchronizes the device. reset != 0 clears it. */
tgs_status tgs_last_device_error(int32_t reset);

/* Sets the limit, in nanoseconds of the device's global timer, of one look-back wait of the bin
 * sort (tgs_bin_sort, tgs_bin_sort_static and the service's binning) for the calls launched after
 * it, process-wide; ns <= 0 restores the default of 1 s. A CUDA graph keeps the limit it was
 * captured with. Returns the previous limit. A limit far below a tile's run time makes waits run
 * out: a way to exercise the time-out path. */
int64_t tgs_set_lookback_limit(int64_t ns);

/* ---------------------------------------------------------------------------------------------
 * Rendering service (tgs_serve_*): resident scenes and asynchronous frame requests.
 *
 * A server owns device copies of its scenes, `slots` sets of frame buffers and a worker thread.
 * Every buffer is allocated by tgs_serve_create (slots) and tgs_serve_add_scene (scenes), charged
 * to hbm_budget_bytes; the worker allocates nothing. A request enters a free slot in submission
 * order and is preprocessed and binned there (the calls above, on the slot's own stream), so
 * requests of different scenes and resolutions overlap on the GPU. With a tensor-core precision
 * the worker then rasterizes every binned request together in ONE persistent launch
 * (tgs_rasterize_batch; at most two launches in flight), so requests that arrive while a launch
 * runs are binned meanwhile and join the next one (continuous batching); with FP32 each slot
 * rasterizes on its own stream. The batched launch waits (bounded, 2 s) on a per-slot device
 * readiness flag; every slot has its own device status word, so a time-out in one frame is
 * reported for that request only.
 *
 * Requests are identified by tickets. A ticket's record is released when poll or wait reports it
 * done; later calls with it return TGS_ERR_NOT_FOUND. Waits are bounded: tgs_serve_wait returns
 * TGS_ERR_TIMEOUT after timeout_ms, and a request not finished within request_timeout_ms (if > 0)
 * completes with TGS_ERR_TIMEOUT (its slot is reused once the GPU has finished its work).
 * Functions may be called from any host thread; a server must not be used after destroy. */

typedef struct {
  int64_t hbm_budget_bytes;   /* device bytes the server may hold (scenes + slot buffers) */
  int32_t max_inflight;       /* queued + rendering requests admitted at once (>= 1) */
  int32_t slots;              /* frames in flight (1..16), each with its own buffers */
  int32_t device;             /* CUDA device ordinal (must be sm_103) */
  int32_t precision;          /* TGS_PRECISION_* */
  tgs_tiling tiling;          /* tile grouping (and binning flags) of every frame; the tensor-core
                                 precisions take 1x1, 2x2, 4x2, 2x4 or 4x4 groups */
  float bg[3];                /* background colour */
  int32_t request_timeout_ms; /* 0 = no limit */
  int64_t max_gaussians;      /* largest scene a slot renders (1 .. 2^30 - 1) */
  int32_t max_width, max_height; /* largest frame a slot renders (1 .. 16384 each) */
  int64_t max_entries;        /* bin entries a frame may need (1 .. 2^30 - 1); a frame that needs
                                 more completes with TGS_ERR_CAPACITY */
} tgs_serve_config;

typedef struct tgs_server tgs_server; /* opaque */

#define TGS_SERVE_MAX_RESOLUTIONS 16
typedef struct {
  int32_t width, height;
  int64_t completed;          /* requests of this resolution completed with TGS_OK */
  double mean_ms, p50_ms, p99_ms; /* submit -> completion latency over the last 4096 of them */
} tgs_serve_resolution_stats;

typedef struct {
  int64_t submitted;          /* admitted requests */
  int64_t rejected;           /* submissions refused with TGS_ERR_BUSY */
  int64_t completed;          /* requests completed with TGS_OK */
  int64_t failed;             /* requests completed with an error (including time-outs) */
  int64_t regrown;            /* unused (0): slot capacities are fixed at creation */
  int64_t inflight;           /* queued + rendering now */
  int64_t hbm_bytes;          /* device bytes held by the server now */
  double seconds;             /* since tgs_serve_create */
  double frames_per_second;   /* completed / seconds */
  int32_t num_resolutions;
  tgs_serve_resolution_stats res[TGS_SERVE_MAX_RESOLUTIONS]; /* in order of first appearance */
} tgs_serve_stats;

/* Creates a server, its slot buffers (sized by the max_* fields) and its worker thread on
 * config->device. INVALID_ARGUMENT for a bad config, CAPACITY if the slot buffers exceed the
 * budget, UNSUPPORTED_DEVICE if the device is not sm_103, CUDA if an allocation or a stream fails. */
tgs_status tgs_serve_create(const tgs_serve_config* config, tgs_server** out);

/* Copies a scene (the arrays of `scene` may be host or device memory) into server-owned device
 * memory and returns its id. CAPACITY if the copy would exceed the budget or the scene has more
 * than max_gaussians Gaussians. Synchronous. */
tgs_status tgs_serve_add_scene(tgs_server* server, const tgs_scene* scene, int32_t* scene_id);

/* Frees a scene. BUSY while admitted requests use it, NOT_FOUND for an unknown id. */
tgs_status tgs_serve_remove_scene(tgs_server* server, int32_t scene_id);

/* Admits a request to render `scene_id` from `camera` into out_rgb (device [3,H,W] planar) and,
 * if non-NULL, out_T (device [H,W]); both are caller-owned and must stay valid until the request
 * is done. Returns at once with a ticket. BUSY if max_inflight requests are admitted already;
 * NOT_FOUND for an unknown scene; INVALID_ARGUMENT for a bad camera or NULL out_rgb. A request
 * larger than max_width x max_height, or whose frame needs more than max_entries bin entries,
 * completes with CAPACITY. */
tgs_status tgs_serve_submit(tgs_server* server, int32_t scene_id, const tgs_camera* camera,
                            float* out_rgb, float* out_T, uint64_t* ticket);

/* Non-blocking: *done = 1 and *result = the request's status if it has completed (the ticket is
 * then released), else *done = 0. NOT_FOUND for an unknown ticket. */
tgs_status tgs_serve_poll(tgs_server* server, uint64_t ticket, int32_t* done, tgs_status* result);

/* Blocks until the request completes (then as poll) or timeout_ms passes (TGS_ERR_TIMEOUT, the
 * ticket stays valid). */
tgs_status tgs_serve_wait(tgs_server* server, uint64_t ticket, int32_t timeout_ms,
                          tgs_status* result);

/* Pause (paused != 0) or resume moving queued requests into slots. Frames already in slots
 * finish; submissions are still admitted up to max_inflight. */
tgs_status tgs_serve_pause(tgs_server* server, int32_t paused);

tgs_status tgs_serve_get_stats(tgs_server* server, tgs_serve_stats* out);

/* Stops the worker, waits (bounded) for the frames in slots, frees all device memory and the
 * server. Requests still queued are dropped. */
tgs_status tgs_serve_destroy(tgs_server* server);

/* ---------------------------------------------------------------------------------------------
 * Frame sequences from host memory (tgs_frames_*): a scene in host memory rendered from a list of
 * cameras into host images, every frame the Section 2 pipeline (tgs_preprocess -> tgs_bin_sort ->
 * tgs_rasterize), with the host <-> device copies overlapped with the frames' kernels.
 *
 * A tgs_frames object owns two device copies of a scene, `sets` buffer sets (projected
 * attributes, bins with their workspace, one image) and its streams: one for uploads, one per
 * buffer set for preprocess + bin sort (of the highest priority), one for rasterization (frames in
 * order) and one for downloads. Each call uploads the scene into the copy the previous call did
 * not use, so one call's upload overlaps the previous call's frames; frame k of a call takes
 * buffer set (frames enqueued before it) % sets, which is reused once its image has been
 * downloaded. Every buffer is allocated by tgs_frames_create; the calls allocate nothing. An
 * object is used by one host thread at a time and must not be used after destroy. */

typedef struct {
  int64_t max_gaussians;         /* largest scene (1 .. 2^30 - 1) */
  int32_t max_sh_degree;         /* largest SH degree of a scene (0..3) */
  int32_t max_width, max_height; /* largest frame (1 .. 16384 each) */
  int64_t max_entries;           /* bin entries a frame may need (1 .. 2^30 - 1); a frame that needs
                                    more renders the background and tgs_frames_wait reports
                                    TGS_ERR_CAPACITY */
  tgs_tiling tiling;             /* tile grouping (and binning flags) of every frame; the tensor-core
                                    precisions take 1x1, 2x2, 4x2, 2x4 or 4x4 groups */
  int32_t precision;             /* TGS_PRECISION_* */
  float bg[3];                   /* background colour */
  int32_t sets;                  /* buffer sets = frames in flight (2..8) */
  int32_t device;                /* CUDA device ordinal (must be sm_103) */
} tgs_frames_config;

typedef struct tgs_frames tgs_frames; /* opaque */

/* Allocates the object's device buffers (on config->device) and streams. INVALID_ARGUMENT for a
 * bad config, UNSUPPORTED_DEVICE off sm_103, CUDA when an allocation fails (nothing is kept). */
tgs_status tgs_frames_create(const tgs_frames_config* config, tgs_frames** out);

/* Device bytes the object holds. */
int64_t tgs_frames_device_bytes(const tgs_frames* frames);

/* Enqueues one call and returns: the upload of `scene` (host arrays, [n,...] as tgs_scene; page-
 * locked memory makes the copies asynchronous), then for every camera k (all of one size) the
 * frame's kernels and the download of its image into out_rgb + k * 3 * H * W (host, [count,3,H,W])
 * and, if out_T != NULL, of its transmittance into out_T + k * H * W. The host arrays must stay
 * untouched until the call has completed: tgs_frames_wait, or work enqueued afterwards on `stream`
 * (which is made to wait for the call; NULL = the default stream). INVALID_ARGUMENT for NULL
 * pointers, a scene or frame larger than the config's, cameras of different sizes, count < 0;
 * count = 0 does nothing. A launch that fails ends the call with its status after the frames
 * before it; the call's events are still recorded, so later calls and `stream` are ordered after
 * everything it enqueued. */
tgs_status tgs_frames_render(tgs_frames* frames, const tgs_scene* scene, const tgs_camera* cams,
                             int32_t count, float* out_rgb, float* out_T, void* stream);

/* Blocks until every call enqueued so far has completed. Returns TGS_ERR_CAPACITY if a frame since
 * the last wait needed more than max_entries bin entries (its image is the background),
 * TGS_ERR_TIMEOUT if a bounded wait of the bin sort ran out (that frame's bins were empty), else
 * TGS_OK; the conditions are cleared. Time-outs of the rasterizer's own waits are reported by
 * tgs_last_device_error, as for tgs_rasterize. */
tgs_status tgs_frames_wait(tgs_frames* frames);

/* Waits for the object's work, then frees its buffers, streams and the object. */
tgs_status tgs_frames_destroy(tgs_frames* frames);

#ifdef __cplusplus
}
#endif
#endif /* TGS_H */
