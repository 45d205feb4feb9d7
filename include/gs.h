/*
 * gs.h - C ABI of the GB300 (sm_103a) differentiable tile-based Gaussian
 * splatting library (libgs_gb300.so).
 *
 * The library implements the per-step operators of Gaussian-splatting
 * training that arXiv 2606.11390 distributes across GPUs (§4 "Distributed
 * Gaussian Splatting"): per-Gaussian spherical-harmonic colour evaluation and
 * projection, which yield a colour and projected geometry per camera of the
 * batch; a depth sort per camera; tile rasterisation; and the backward pass of
 * each, which sums per-Gaussian gradients with atomics. The paper takes
 * the mathematics of these operators from 3D Gaussian Splatting (Kerbl et al.
 * 2023, cited in §1): EWA projection of 3D Gaussians, real SH colour of degree
 * <= 3, and front-to-back alpha compositing of depth-sorted splats per tile.
 * Everything here runs on one GPU.
 *
 * Conventions common to every entry point
 * ---------------------------------------
 * - Pointers named *_dev or documented as "device" point to device memory;
 *   everything else is host memory. All device buffers are allocated and
 *   owned by the caller. The library never allocates or frees memory and
 *   never synchronises the device or the stream: every call only enqueues
 *   work on `stream` (a cudaStream_t; NULL means the legacy default stream)
 *   and returns.
 * - Return value: GS_OK, or a synchronous error found before or while
 *   enqueuing (bad argument, unsupported configuration, CUDA launch error).
 *   On a synchronous error nothing has been enqueued unless the code is
 *   GS_ERR_CUDA.
 * - Conditions only known on the device are OR-ed as GS_STATUS_* bits into
 *   the caller's int32 device word `status_dev`; the caller reads it after the
 *   stream has completed and clears it when it wants to.
 * - Float arrays are IEEE binary32. Device pointers must be 16-byte aligned
 *   (cudaMalloc and PyTorch allocations are); gs_project and gs_rasterize_bwd
 *   use TMA bulk copies when they are, and plain loads otherwise.
 *
 * Data layout (N Gaussians, V views, view v is W_v x H_v pixels)
 * ----------------------------------------------------------------
 *   means [N][3], log_scales [N][3], quats [N][4] as (w, x, y, z), not
 *   necessarily normalised, opacity_logits [N], sh [N][16][3]
 *   (coefficient-major, channel-minor; coefficients beyond (degree+1)^2 are
 *   ignored).
 *   cams_dev: V gs_camera records in device memory (poses and intrinsics).
 *   sizes: V pairs (W_v, H_v) in host memory; they fix the tile and pixel
 *   layout of a call.
 *   Record index of (view v, Gaussian g) is vg = v*N + g.
 *   Tiles: view v has ntx_v = ceil(W_v / tile_w) by nty_v = ceil(H_v / tile_h)
 *   tiles; the global tile id of (v, tx, ty) is tile_base_v + ty*ntx_v + tx,
 *   with tile_base_v the number of tiles of the views before v.
 *   Pixels: view v's pixels start at pix_base_v = sum_{u<v} W_u H_u and are
 *   row-major; image arrays hold 3 interleaved channels per pixel.
 */
#ifndef GS_GB300_H_
#define GS_GB300_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* gs_stream_t; /* identical to cudaStream_t */

/* Symbol visibility: the library is built with hidden visibility and exports
 * exactly the functions declared with GS_API. */
#if defined(__GNUC__)
#define GS_API __attribute__((visibility("default")))
#else
#define GS_API
#endif

/* Synchronous return codes. */
#define GS_OK 0
#define GS_ERR_ARG 1         /* invalid argument (null pointer, bad size, misaligned, ...) */
#define GS_ERR_CUDA 2        /* a CUDA call failed while enqueuing */
#define GS_ERR_UNSUPPORTED 3 /* valid but unsupported configuration (tile size, view count) */
#define GS_ERR_TOO_LARGE 4   /* the problem needs more scratch than gs_bin_sort_static has */

/* Asynchronous status bits, OR-ed into *status_dev. */
#define GS_STATUS_CAPACITY 1 /* more tile intersections than `capacity`: keys clipped, ranges invalid */
#define GS_STATUS_TIMEOUT 2  /* a bounded device-side wait gave up: results of that call are invalid */
#define GS_STATUS_BOUNDS 4   /* an index failed a device-side range check and was skipped */

#define GS_MAX_VIEWS 64

/* One camera, 80 bytes. viewmat is the row-major 4x4 world->camera matrix in
 * OpenCV axes (+x right, +y down, +z forward); fx, fy, cx, cy in pixels. */
typedef struct gs_camera {
  float viewmat[16];
  float fx, fy, cx, cy;
} gs_camera;

/* Rendering constants, 60 bytes. tile_w x tile_h must be one of 8x8, 16x16,
 * 32x16, 32x32. sh_degree in 0..3. flags: GS_FLAG_* bits. Culling: near_plane < depth < far_plane. eps2d is
 * added to the diagonal of every 2D covariance. Compositing: alpha =
 * min(alpha_cap, opacity * exp(-power)); entries with alpha < alpha_min are
 * skipped; compositing stops before the entry that would take the
 * transmittance below t_stop. bg is added with the final transmittance.
 * raster_batch_fwd / raster_batch_bwd: splats the rasteriser stages per
 * shared-memory batch in the forward / backward, 0 for the default
 * (forward: max(threads per tile, 128); backward: threads per tile, clamped
 * to [64, 256]) or one of 64, 128, 256, 512 (GS_ERR_UNSUPPORTED otherwise;
 * a backward batch whose staging exceeds 48 KB of shared memory, as 512 on
 * tiles of more than 4 warps, is launched with the opt-in for more); a
 * performance choice only, results are the same (with a
 * non-zero bg the backward keeps its default). Threads per tile = tile_w *
 * tile_h / pixels per thread (see GS_FLAG_RASTER_2PX). */
typedef struct gs_config {
  int32_t tile_w, tile_h, sh_degree, flags;
  float near_plane, far_plane, eps2d, alpha_cap, alpha_min, t_stop;
  float bg[3];
  int32_t raster_batch_fwd, raster_batch_bwd;
} gs_config;

/* gs_config.flags: gs_rasterize_bwd adds the parameter gradients to the
 * output arrays instead of overwriting them (to sum over separate calls). */
#define GS_FLAG_ACCUMULATE_GRADS 1
/* gs_config.flags: the rasteriser gives each thread 2 pixels (8-column warp
 * blocks) instead of 4 (16-column warp blocks) for 16x16, 32x16 and 32x32 tiles;
 * a performance choice only, results are the same. */
#define GS_FLAG_RASTER_2PX 2
/* gs_config.flags, test hook for the bounded device waits: in gs_bin_sort the
 * first tile of the first depth pass withholds its prefix, so the next tile's
 * look-back runs out its (here shortened) iteration bound and the call
 * reports GS_STATUS_TIMEOUT; its outputs are then invalid but every access
 * stays in bounds and the context stays usable. Never set in normal use. */
#define GS_FLAG_TEST_STALL_LOOKBACK 4
/* gs_config.flags: tile scheduling order. With this flag `tile_ranges` holds
 * n_tiles x 3 uint32: the [n_tiles][2] ranges followed by a permutation of
 * the tile ids, longest list first (by half-octaves of the list length),
 * which gs_bin_sort writes and the rasteriser follows when it hands tiles to
 * CTAs: the heavy tiles start first and do not form the tail of the launch.
 * Results are the same with or without it. */
#define GS_FLAG_TILE_ORDER 8

/* Number of 32-bit floats in one projected record (see gs_project). */
#define GS_RECORD_FLOATS 12
/* Number of 32-bit floats of gradient per projected record (see gs_rasterize_bwd). */
#define GS_DRECORD_FLOATS 9

/* Library version (major*10000 + minor*100 + patch). */
GS_API int gs_version(void);

/* Human-readable text for a synchronous return code (GS_OK, GS_ERR_*). Never NULL. */
GS_API const char* gs_status_string(int code);

/* Tile and pixel totals of a view layout (host only, nothing enqueued).
 * sizes: V (W, H) pairs, host. Writes *n_tiles and *n_pixels (either may be
 * NULL). Errors: GS_ERR_ARG for V outside 1..GS_MAX_VIEWS or non-positive
 * sizes; GS_ERR_UNSUPPORTED for a tile size other than 8x8, 16x16, 32x16,
 * 32x32. */
GS_API int gs_layout_totals(const int32_t* sizes, int32_t V, const gs_config* cfg, int64_t* n_tiles, int64_t* n_pixels);

/* gs_project - per-(view, Gaussian) SH colour and EWA projection.
 * Paper: §4, the spherical-harmonics and projection operators, which compute
 * per Gaussian its colour and projected geometry for every camera of the
 * batch; mathematics of 3DGS (Kerbl et al. 2023): s = exp(log_scale), q/|q|,
 * opacity = sigmoid(logit), Sigma = R S S R^T, t = W mean + t_cam,
 * Sigma2 = J W Sigma W^T J^T + eps2d I with the pinhole Jacobian J at t (frustum
 * clamped to 1.3x the field of view), conic = Sigma2^-1, 3-sigma radius from
 * the larger eigenvalue, tile rectangle, colour = max(0, SH(dir) + 0.5).
 * One launch covers all V views (parameters are read once per Gaussian).
 *
 * in  (device): means, log_scales, quats, opacity_logits, sh; cams_dev [V].
 * in  (host)  : sizes [V][2], cfg.
 * out (device): projected [V*N][12] floats per record vg:
 *                 0 mean2d.x  1 mean2d.y  2 conic A  3 conic B  4 conic C
 *                 5 opacity   6 depth     7 radius   8 r  9 g  10 b  11 = 0
 *               (all zero for an invisible record);
 *               rects [V*N][4] int16 tile rectangle (x0, y0, x1, y1), half-open;
 *               counts [V*N] uint32 = (x1-x0)*(y1-y0), 0 if culled;
 *               depth_keys [V*N] uint32 (optional, NULL to skip): the float
 *               bits of the depth (field 6) of a visible record, 0 for a
 *               culled one. gs_bin_sort reads them instead of gathering the
 *               depths from the 48-byte records.
 * N may be 0 (nothing enqueued). Errors: GS_ERR_ARG, GS_ERR_UNSUPPORTED, GS_ERR_CUDA. */
GS_API int gs_project(const float* means, const float* log_scales, const float* quats, const float* opacity_logits,
               const float* sh, int64_t N, const gs_camera* cams_dev, const int32_t* sizes, int32_t V,
               const gs_config* cfg, float* projected, int16_t* rects, uint32_t* counts, uint32_t* depth_keys,
               int32_t* status_dev, gs_stream_t stream);

/* Bytes of device workspace gs_bin_sort needs for N Gaussians, V views, a
 * key capacity and n_tiles tiles (from gs_layout_totals); 0 for invalid
 * arguments. About 16 V N + 18 capacity + 276 n_tiles bytes. */
GS_API size_t gs_bin_sort_workspace_bytes(int64_t N, int32_t V, int64_t capacity, int64_t n_tiles);

/* gs_bin_sort - tile keys and per-camera depth sort.
 * Paper: §4, where each camera's Gaussians are depth-sorted before
 * rasterisation, and §3.2 (the paper sorts with CUB's radix sort; this is a
 * CUB-free onesweep LSD radix sort). Result: for every visible record vg
 * (views ascending, Gaussians ascending) and every tile (tx, ty) of its
 * rectangle in row-major order one pair
 *   key = (global tile id << 32) | float bits of depth,  val = vg,
 * stably sorted by key, so equal keys stay in record-index order; and
 * tile_ranges[t] = [start, end) of tile t's entries in the sorted list
 * ([0, 0) for an empty tile). Computed as a depth sort of the visible records,
 * a stable binning of them into super-tiles of 8 x 8 tiles, and a placement
 * of each record in the lists of the tiles it covers in that order, which
 * yields the same order.
 *
 * in  (device): projected, rects, counts from gs_project; depth_keys from
 *               gs_project (optional: with NULL the depths are read from the
 *               projected records; the result is the same).
 * in  (host)  : N, sizes [V][2], cfg, capacity (>= 0, < 2^32 - 1).
 * out (device): vals [capacity] uint32 (first n entries valid);
 *               keys [capacity] uint64 (optional: pass NULL to skip writing
 *               the 64-bit keys; nothing downstream needs them);
 *               tile_ranges [n_tiles][2] uint32;
 *               n_isect_dev [1] int64 = total number of intersections.
 * workspace (device, caller-owned, >= gs_bin_sort_workspace_bytes, 256-byte
 *   aligned): scratch, contents undefined on return.
 * If the total exceeds `capacity`, GS_STATUS_CAPACITY is set, no write goes
 * past `capacity`, and keys, vals and ranges are incomplete and must not be
 * used: grow the buffers to *n_isect_dev (always the exact total) and call
 * again. A device wait that exceeds its iteration bound sets
 * GS_STATUS_TIMEOUT.
 * Errors: GS_ERR_ARG (also for a too-small workspace), GS_ERR_CUDA. */
GS_API int gs_bin_sort(const float* projected, const int16_t* rects, const uint32_t* counts, const uint32_t* depth_keys,
                int64_t N, const int32_t* sizes, int32_t V, const gs_config* cfg, uint64_t* keys, uint32_t* vals,
                int64_t capacity,
                uint32_t* tile_ranges, int64_t* n_isect_dev, void* workspace, size_t workspace_bytes,
                int32_t* status_dev, gs_stream_t stream);

/* gs_bin_sort_partitioned_workspace_bytes - workspace of
 * gs_bin_sort_partitioned; 0 for invalid arguments (partitions not a power of
 * two in [1, 64]). */
GS_API size_t gs_bin_sort_partitioned_workspace_bytes(int64_t N, int32_t V, int64_t capacity, int64_t n_tiles,
                                                      int32_t partitions);

/* gs_bin_sort_partitioned - gs_bin_sort with its depth sort run the way the
 * paper sorts across devices (§4): the V*N records are split into
 * `partitions` contiguous ranges, each range is compacted and depth-sorted on
 * its own, and the sorted ranges are combined by a log2(partitions)-level
 * merge tree in which every output block finds its split of the two input
 * runs by a merge-path binary search. Here the partitions share one GPU (an
 * emulation of the multi-device sort); the result is identical, bit for bit,
 * to gs_bin_sort's. Arguments as gs_bin_sort, plus partitions (a power of two
 * in [1, 64]) and a workspace of gs_bin_sort_partitioned_workspace_bytes.
 * Errors: as gs_bin_sort. */
GS_API int gs_bin_sort_partitioned(const float* projected, const int16_t* rects, const uint32_t* counts,
                                   const uint32_t* depth_keys, int64_t N, const int32_t* sizes, int32_t V,
                                   const gs_config* cfg, uint64_t* keys,
                                   uint32_t* vals, int64_t capacity, uint32_t* tile_ranges, int64_t* n_isect_dev,
                                   int32_t partitions, void* workspace, size_t workspace_bytes, int32_t* status_dev,
                                   gs_stream_t stream);

/* gs_bin_sort_static - gs_bin_sort without a caller-provided workspace.
 * The paper has no counterpart: this variant exists for callers that cannot
 * allocate device memory where they sort (plug-ins whose host application
 * owns every device allocation, services that forbid allocation after
 * start-up, threads that must not risk cudaMalloc's device synchronisation).
 * It allocates nothing; its scratch is one file-scope device array of
 * GS_STATIC_SCRATCH_BYTES (64 MiB) that each GPU loading this code holds
 * until the process exits.
 * Arguments, outputs and status bits are those of gs_bin_sort, minus the
 * workspace and the optional depth keys (the depths are read from the
 * projected records). Limit: gs_bin_sort_workspace_bytes(N, V, capacity, n_tiles)
 * must not exceed GS_STATIC_SCRATCH_BYTES (about 16 V N + 18 capacity + 276 n_tiles bytes),
 * else GS_ERR_TOO_LARGE is returned and nothing is enqueued.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.
 * All calls share the one array, which keeps the last call's contents (the
 * parts that must start at zero are cleared by every call): calls that can
 * overlap on the GPU (different streams, or several threads) race with each
 * other and must be serialised by the caller. */
#define GS_STATIC_SCRATCH_BYTES (64u << 20)
GS_API int gs_bin_sort_static(const float* projected, const int16_t* rects, const uint32_t* counts, int64_t N,
                              const int32_t* sizes, int32_t V, const gs_config* cfg, uint64_t* keys, uint32_t* vals,
                              int64_t capacity, uint32_t* tile_ranges, int64_t* n_isect_dev, int32_t* status_dev,
                              gs_stream_t stream);

/* gs_rasterize_fwd - tile rasterisation (front-to-back alpha compositing).
 * Paper: §4, the rasterisation operator that renders each camera's image;
 * rule of 3DGS: for pixel p (sampled at its centre) of tile t, for the
 * entries of t in sorted order, power = 0.5 d^T conic d with d = p - mean2d,
 * skip if power < 0, alpha = min(alpha_cap, opacity exp(-power)), skip if
 * alpha < alpha_min, stop before the entry whose T(1-alpha) < t_stop, else
 * C += colour alpha T and T *= (1 - alpha). out = C + T bg.
 *
 * in  (device): projected, vals (sorted), tile_ranges from gs_bin_sort.
 * in  (host)  : sizes [V][2], cfg.
 * out (device): image [P][3], final_T [P] (transmittance after the last
 *               composited entry), last [P] uint32 (1 + position, within its
 *               tile's range, of the last composited entry; 0 if none).
 * cull_masks (device, optional, [capacity] uint16 like vals, 2-byte aligned;
 *               NULL for none): for every list entry the kernel stages, the
 *               warps of its tile whose pixel block the splat can reach,
 *               tagged with the warp layout (tile shape, pixels per thread),
 *               for gs_rasterize_bwd / gs_rasterize_bwd_pixels on the same
 *               lists to reuse instead of recomputing; other entries are left
 *               as they were. Not written for 32x32 tiles at 2 pixels per
 *               thread. A performance aid only: the backward's results are
 *               the same with or without it.
 * Errors: GS_ERR_ARG, GS_ERR_UNSUPPORTED, GS_ERR_CUDA. */
GS_API int gs_rasterize_fwd(const float* projected, const uint32_t* vals, const uint32_t* tile_ranges, const int32_t* sizes,
                     int32_t V, const gs_config* cfg, float* image, float* final_T, uint32_t* last,
                     uint16_t* cull_masks, gs_stream_t stream);

/* gs_rasterize_fwd_counted - gs_rasterize_fwd (same outputs) that also counts
 * the pixel-splat pairs of its work, for measuring the rasteriser against its
 * arithmetic roofline (paper §4 names rasterisation the cost centre of the
 * step). A separately compiled variant of the kernel: the normal entry points
 * count nothing.
 * out (device): pair_counts_dev [3] uint64, added to (the caller zeroes it):
 *   [0] pairs executed: for every splat a warp takes from its tile's list
 *       after its per-warp cull, one pair per pixel of each thread that runs
 *       the step (pixels that have stopped or lie outside the image included);
 *   [1] pairs evaluated: those of [0] whose pixel is still compositing;
 *   [2] pairs composited: those of [1] with power >= 0, alpha >= alpha_min
 *       and T (1 - alpha) >= t_stop.
 * Errors: as gs_rasterize_fwd; GS_ERR_ARG for a null or misaligned
 * pair_counts_dev. */
GS_API int gs_rasterize_fwd_counted(const float* projected, const uint32_t* vals, const uint32_t* tile_ranges,
                                    const int32_t* sizes, int32_t V, const gs_config* cfg, float* image,
                                    float* final_T, uint32_t* last, uint64_t* pair_counts_dev, uint16_t* cull_masks,
                                    gs_stream_t stream);

/* gs_rasterize_fwd_l1l2 - gs_rasterize_fwd with the L1 + L2 image loss of
 * gs_image_loss computed in the same kernel, as each pixel's colour is final
 * (the rendered image is not read back). Paper: §4, rasterisation and the
 * per-camera image loss; the loss is the workloads' L = w_l1 mean|r| +
 * w_l2 mean(r^2), r = image - target, means over n_values values.
 * in  (device): as gs_rasterize_fwd; target [P][3] laid out like image.
 * in  (host)  : as gs_rasterize_fwd; n_values (>= 3 P; the total over all
 *               calls whose losses add up, e.g. all views rendered one call
 *               per view); accumulate (0: loss_dev is zeroed first, else the
 *               call adds to it).
 * out (device): image, final_T, last as gs_rasterize_fwd; dL_dimage [P][3]
 *               = (w_l1 sign(r) + 2 w_l2 r) / n_values, bit-identical to
 *               gs_image_loss's; loss_dev [1] double += this call's sum of
 *               (w_l1 |r| + w_l2 r^2) / n_values (atomic adds: the last bits
 *               depend on their order); cull_masks as gs_rasterize_fwd.
 * Errors: GS_ERR_ARG (also n_values < 3 P), GS_ERR_UNSUPPORTED, GS_ERR_CUDA. */
GS_API int gs_rasterize_fwd_l1l2(const float* projected, const uint32_t* vals, const uint32_t* tile_ranges,
                                 const int32_t* sizes, int32_t V, const gs_config* cfg, float* image, float* final_T,
                                 uint32_t* last, const float* target, int64_t n_values, float w_l1, float w_l2,
                                 int32_t accumulate, float* dL_dimage, double* loss_dev, uint16_t* cull_masks,
                                 gs_stream_t stream);

/* gs_rasterize_bwd - backward of rasterisation, projection and SH colour.
 * Paper: §4, where the backward pass keeps the forward pass's partitioning
 * and sums gradients with atomics; here device-scope FP32 atomics on one
 * GPU. Each pixel walks its tile's list in
 * reverse from `last`, recovering the transmittance before each entry from
 * final_T by dividing by (1 - alpha) instead of storing per-pixel lists.
 * Per-entry gradients are reduced across each warp with shuffles, summed per
 * tile in shared memory and added to d_projected with one atomic per value.
 * A second kernel then chains d_projected through colour, conic, 2D mean,
 * Jacobian, view transform, covariance and the activations to the parameter
 * gradients, one thread per Gaussian summing over views (no atomics).
 * Equivalent to gs_rasterize_bwd_pixels followed by gs_project_bwd.
 *
 * in  (device): the parameters and cams_dev given to gs_project; projected,
 *               counts from gs_project; vals, tile_ranges from gs_bin_sort;
 *               final_T, last from gs_rasterize_fwd; dL_dimage [P][3].
 * in  (host)  : N, sizes [V][2], cfg.
 * scratch/out (device): d_projected [V*N][9] = dL/d(mean2d.x, mean2d.y,
 *               conic A, B, C, r, g, b, opacity) per record; zeroed by this
 *               call, then accumulated.
 * out (device): d_means [N][3], d_log_scales [N][3], d_quats [N][4],
 *               d_opacity_logits [N], d_sh [N][16][3]: overwritten, or added
 *               to when cfg->flags has GS_FLAG_ACCUMULATE_GRADS; d_sh
 *               coefficients beyond the degree receive 0.
 * in  (device, optional): cull_masks written by the forward on the same lists
 *               (NULL: the backward computes the cull itself; an entry whose
 *               tag does not match this call's warp layout is recomputed).
 * Errors: GS_ERR_ARG, GS_ERR_UNSUPPORTED, GS_ERR_CUDA. */
GS_API int gs_rasterize_bwd(const float* means, const float* log_scales, const float* quats, const float* opacity_logits,
                     const float* sh, int64_t N, const gs_camera* cams_dev, const int32_t* sizes, int32_t V,
                     const gs_config* cfg, const float* projected, const uint32_t* counts, const uint32_t* vals,
                     const uint32_t* tile_ranges, const float* final_T, const uint32_t* last, const float* dL_dimage,
                     float* d_projected, float* d_means, float* d_log_scales, float* d_quats, float* d_opacity_logits,
                     float* d_sh, const uint16_t* cull_masks, int32_t* status_dev, gs_stream_t stream);

/* gs_rasterize_bwd_pixels - first half of gs_rasterize_bwd: the per-pixel
 * reverse compositing only. Zeroes d_projected [V*N][9] (device) and
 * accumulates into it dL/d(mean2d, conic, colour, opacity) of every record;
 * the other arguments are those of gs_rasterize_bwd.
 * Errors: GS_ERR_ARG, GS_ERR_UNSUPPORTED, GS_ERR_CUDA. */
GS_API int gs_rasterize_bwd_pixels(const float* projected, const uint32_t* vals, const uint32_t* tile_ranges,
                                   const int32_t* sizes, int32_t V, const gs_config* cfg, int64_t N,
                                   const float* final_T, const uint32_t* last, const float* dL_dimage,
                                   float* d_projected, const uint16_t* cull_masks, gs_stream_t stream);

/* gs_rasterize_bwd_pixels_counted - gs_rasterize_bwd_pixels (same outputs)
 * that also counts the pixel-splat pairs of its work (paper §4, the backward
 * of rasterisation), like gs_rasterize_fwd_counted:
 * out (device): pair_counts_dev [3] uint64, added to (the caller zeroes it):
 *   [0] pairs executed (listed splats x pixels of each thread running the
 *       step), [1] pairs evaluated: those of [0] whose entry lies before the
 *       pixel's last contributor, [2] pairs composited in the forward among
 *       [1] (the ones that receive a gradient).
 * Errors: as gs_rasterize_bwd_pixels; GS_ERR_ARG for a null or misaligned
 * pair_counts_dev. */
GS_API int gs_rasterize_bwd_pixels_counted(const float* projected, const uint32_t* vals,
                                           const uint32_t* tile_ranges, const int32_t* sizes, int32_t V,
                                           const gs_config* cfg, int64_t N, const float* final_T,
                                           const uint32_t* last, const float* dL_dimage, float* d_projected,
                                           uint64_t* pair_counts_dev, const uint16_t* cull_masks,
                                           gs_stream_t stream);

/* gs_project_bwd - second half of gs_rasterize_bwd: chains d_projected
 * (from gs_rasterize_bwd_pixels) through SH colour and projection to the
 * parameter gradients, one thread per Gaussian summing over views. Outputs
 * and flags as in gs_rasterize_bwd. Errors: GS_ERR_ARG, GS_ERR_UNSUPPORTED,
 * GS_ERR_CUDA. */
GS_API int gs_project_bwd(const float* means, const float* log_scales, const float* quats, const float* opacity_logits,
                          const float* sh, int64_t N, const gs_camera* cams_dev, const int32_t* sizes, int32_t V,
                          const gs_config* cfg, const uint32_t* counts, const float* d_projected, float* d_means,
                          float* d_log_scales, float* d_quats, float* d_opacity_logits, float* d_sh,
                          int32_t* status_dev, gs_stream_t stream);

/* gs_image_loss - image-space loss and its gradient.
 * Paper: §4 names an image-space loss per camera (fused SSIM); this is the
 * L1 + L2 loss of the workloads: L = w_l1 mean|r| + w_l2 mean(r^2),
 * r = image - target, means over all n values.
 * in  (device): image [n], target [n]. out (device): dL_dimage [n]
 * (overwritten), loss_dev [1] double (overwritten). Errors: GS_ERR_ARG, GS_ERR_CUDA. */
GS_API int gs_image_loss(const float* image, const float* target, int64_t n, float w_l1, float w_l2, float* dL_dimage,
                  double* loss_dev, gs_stream_t stream);

/* gs_ssim_loss - fused SSIM image loss and its gradient, one kernel.
 * Paper: §4 runs a fused SSIM loss operator per camera (SSIM of Wang et al.
 * 2004, fused as in Taming 3DGS). L = (1 - lambda) mean|x - y|
 * + lambda (1 - mean SSIM(x, y)), means over every pixel and channel of all
 * views; SSIM per channel with an 11x11 Gaussian window (sigma 1.5, weights
 * summing to 1), C1 = 0.01^2, C2 = 0.03^2, pixels outside the image taken as
 * zero in every window sum. The usual training weight is lambda = 0.2.
 * in  (device): image, target [P][3] packed by view like the rendered image
 *     (view v: sizes[2v] x sizes[2v+1] pixels, row-major, RGB interleaved).
 * in  (host): sizes [V][2] int32 (width, height), 1 <= V <= 64.
 * out (device): dL_dimage [P][3] (overwritten), loss_dev [1] double
 *     (overwritten). No workspace: each CTA recomputes its halo on chip.
 * Errors: GS_ERR_ARG (null pointer, bad sizes, lambda outside [0, 1]), GS_ERR_CUDA. */
GS_API int gs_ssim_loss(const float* image, const float* target, const int32_t* sizes, int32_t V, float lambda,
                        float* dL_dimage, double* loss_dev, gs_stream_t stream);

/* gs_morton_workspace_bytes - device scratch gs_morton_order needs for N
 * Gaussians (about 12 N bytes plus look-back state). Returns 0 for N < 0. */
GS_API size_t gs_morton_workspace_bytes(int64_t N);

/* gs_morton_order - permutation that orders Gaussians along a 3D Morton curve.
 * Paper: §5.2 Morton-sorts the Gaussians in three dimensions during
 * densification for memory locality in rasterisation (5-10 %).
 * lo/hi = per-axis min/max of the means; q = clamp(floor((x - lo) *
 * (1024 / (hi - lo))), 0, 1023) per axis, each operation a single rounded
 * float operation in that order (q = 0 where hi == lo, and for NaN);
 * code = bits of qx, qy, qz interleaved, x lowest (30 bits); perm = the
 * stable sort of the codes (equal codes keep index order).
 * in  (device): means [N][3] float32.
 * out (device): perm [N] u32 (perm[i] = old index of the i-th Gaussian in
 *     the new order); codes [N] u32, the sorted codes (optional, may be NULL).
 * workspace: gs_morton_workspace_bytes(N) bytes, 256-byte aligned, owned by
 *     the caller; status_dev as for gs_bin_sort (bounded waits).
 * Errors: GS_ERR_ARG (N >= 2^32 - 1, null pointers, short or misaligned
 * workspace), GS_ERR_CUDA. */
GS_API int gs_morton_order(const float* means, int64_t N, uint32_t* perm, uint32_t* codes, void* workspace,
                           size_t workspace_bytes, int32_t* status_dev, gs_stream_t stream);

/* gs_gather_rows - dst[i] = src[perm[i]] for n_rows rows of row_floats
 * floats (applies a gs_morton_order permutation to any per-Gaussian array:
 * parameters, gradients, optimiser moments). The paper has no separate
 * operator for it (§5.2 reindexes during densification).
 * in  (device): src [n][row_floats], perm [n] (values < n_rows; others are
 *     skipped and set GS_STATUS_BOUNDS in *status_dev).
 * out (device): dst [n][row_floats], distinct from src; 16-byte aligned when
 *     row_floats is a multiple of 4 (then rows move as float4).
 * Errors: GS_ERR_ARG, GS_ERR_CUDA. */
GS_API int gs_gather_rows(const float* src, float* dst, int64_t n_rows, int32_t row_floats, const uint32_t* perm,
                          int32_t* status_dev, gs_stream_t stream);

/* gs_densify_stats - densification statistics of one backward pass.
 * Paper: §5.2 densifies (Kerbl et al. 2023) to large Gaussian counts; the
 * decisions use the accumulated screen-space positional gradient and the
 * largest screen-space radius of each Gaussian. For every view v where
 * Gaussian g is visible (counts[v*N+g] > 0):
 *   grad_accum[g] += sqrt((dmx * W_v/2)^2 + (dmy * H_v/2)^2), with (dmx, dmy)
 *                    = dL/dmean2d from d_projected (pixel units; the factors
 *                    give the gradient in normalised device coordinates);
 *   denom[g] += 1;  max_radii[g] = max(max_radii[g], radius in pixels).
 * in  (device): projected [V*N][12], counts [V*N] (gs_project), d_projected
 *     [V*N][9] (gs_rasterize_bwd). in (host): sizes [V][2], 1 <= V <= 64.
 * in/out (device): grad_accum [N], denom [N], max_radii [N] float32,
 *     accumulated (the caller zeroes them when it starts a statistics window).
 * One thread per Gaussian over all views: no atomics, deterministic.
 * Errors: GS_ERR_ARG, GS_ERR_CUDA. */
GS_API int gs_densify_stats(const float* projected, const uint32_t* counts, const float* d_projected, int64_t N,
                            const int32_t* sizes, int32_t V, float* grad_accum, float* denom, float* max_radii,
                            gs_stream_t stream);

/* gs_adam_step - fused Adam update over a flat parameter array.
 * Paper: §3.2 (fused Adam with vectorised loads and stores and
 * transcendental results cached in shared memory); update of Kingma & Ba
 * 2015: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 * in/out (device): param [n], exp_avg [n], exp_avg_sq [n]; in: grad [n],
 * step_dev [1] int32 = t >= 1 (read on the device, so a captured graph
 * sees the current step). Errors: GS_ERR_ARG, GS_ERR_CUDA. */
GS_API int gs_adam_step(float* param, const float* grad, float* exp_avg, float* exp_avg_sq, int64_t n, float lr, float beta1,
                 float beta2, float eps, const int32_t* step_dev, gs_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GS_GB300_H_ */
