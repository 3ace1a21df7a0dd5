/*
 * mvgs.h -- C ABI of the multi-view differentiable Gaussian-splatting
 * rasterizer (sm_103a).
 *
 * The operations follow Choi, Kim & Kim, "Efficient multi-view training for
 * 3D Gaussian Splatting" (ICCV 2025):
 *   - mvgs_render_views          Eq. 1 rendered for a batch of V cameras with
 *                                the preprocessing of the supplement
 *                                ("Rasterization in multi-view training"):
 *                                participation test, projection, duplication
 *                                per tile, sort by (view, tile, depth), one
 *                                block per (tile, view).
 *   - mvgs_render_views_backward reverse-mode derivative of the above; a
 *                                Gaussian seen in several views sums the
 *                                gradients of all of them (Sec. 5.2).
 *   - mvgs_dssim_loss            photometric l1 + D-SSIM (Sec. 3 and the SSIM
 *                                equations of Sec. 5.1.2), per view.
 *   - mvgs_render_views_sampled  thread-efficient partial rendering (Sec.
 *                                5.1.1, Alg. 3): per (tile, view) only an
 *                                index array of sampled pixels is blended.
 *   - mvgs_adc_accumulate        the multi-view densification error metrics
 *                                E_1 and E_2 of Sec. 5.2.2 (norm per pixel /
 *                                per view, then add).
 *
 * Conventions shared by every call
 *   - Pointers named d_* (and all image / parameter / gradient pointers) are
 *     DEVICE pointers owned by the caller.  Camera arrays are HOST arrays.
 *   - The library never allocates device memory.  Calls that need scratch take
 *     a caller-owned `workspace`; the forward writes everything the backward
 *     needs into a caller-owned `state` buffer.  Sizes come from
 *     mvgs_render_layout() / mvgs_dssim_workspace_size().
 *   - Every call is asynchronous on the given CUDA stream, except that
 *     mvgs_render_views synchronises the stream twice to read the number of
 *     visible (Gaussian, view) records and of duplicated keys back to the
 *     host (they size the sorts) -- unless MVGS_FLAG_CAPTURABLE is set.
 *   - Every call returns an mvgs_status; no exception crosses the ABI.
 *     mvgs_last_error() returns a message for the calling thread.
 *   - Float data is IEEE float32.  Images are packed per view: view v
 *     occupies [3 * P_v, 3 * P_{v+1}) of the buffer, P_v = sum_{u<v} H_u W_u,
 *     each view stored channel-major [3, H, W].
 */
#ifndef MVGS_H
#define MVGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* mvgs_stream;  /* a cudaStream_t; NULL = legacy default stream */

typedef enum mvgs_status {
    MVGS_OK = 0,
    MVGS_EINVAL = 1,      /* bad argument: null pointer, V < 1, empty image, bad tile */
    MVGS_ENOSPACE = 2,    /* state or workspace too small, or a capacity exceeded;
                             the needed counts are reported and nothing is rendered */
    MVGS_EOVERFLOW = 3,   /* a count does not fit the index types (keys >= 2^32,
                             records >= 2^31, global tiles >= 2^32, more than
                             4095 tiles along one axis of a view) */
    MVGS_ECUDA = 4,       /* a CUDA launch or copy failed */
    MVGS_EDEVICE = 5      /* a device-side check failed (e.g. a bounded wait expired) */
} mvgs_status;

/* Pinhole camera with OpenCV axes (+x right, +y down, +z forward).
 * viewmat = [R | t], row-major 3x4, maps world points X to camera points
 * R X + t.  campos is the camera centre in world space (used for the
 * view-dependent colour).  Points with camera depth <= near_z are culled.
 * A pixel (x, y) samples the image plane at (x + 0.5, y + 0.5). */
typedef struct mvgs_camera {
    int32_t width, height;
    float fx, fy, cx, cy;
    float viewmat[12];
    float campos[3];
    float near_z;
} mvgs_camera;

/* The 3D Gaussians of Sec. 3: mean mu, scale S = diag(exp(log_scales)),
 * rotation R from the quaternion (w, x, y, z) (normalised inside), opacity
 * o = sigmoid(opacity_logits), colour from real spherical harmonics of
 * degree sh_degree <= 3 (coefficients [n, (d+1)^2, 3]).  Device pointers,
 * float32, contiguous. */
typedef struct mvgs_scene {
    int64_t n;
    int32_t sh_degree;
    int32_t reserved;
    const float* means;          /* [n, 3] */
    const float* log_scales;     /* [n, 3] */
    const float* quats;          /* [n, 4] */
    const float* opacity_logits; /* [n]    */
    const float* sh;             /* [n, (d+1)^2, 3] */
} mvgs_scene;

/* Render settings.  tile_w x tile_h pixels form one tile: the unit the
 * Gaussians are binned and sorted by.  Blending works on warp-sized strips of
 * a tile.  Supported: tile_w 8, 16 or 32 and tile_h 8, 16, 32 or 64.  The rendered
 * image does not depend on the tile size: a pixel blends a Gaussian only when
 * it lies within the Gaussian's radius on both axes, and every tile that
 * holds such a pixel lists the Gaussian. */
typedef struct mvgs_config {
    int32_t tile_w, tile_h;
    float bg[3];      /* background colour added with the final transmittance */
    uint32_t flags;   /* MVGS_FLAG_* bits below (0 = none) */
    int32_t pixels_per_thread;  /* blend lanes each own this many pixels of a
                                   pixel column, so one warp blends a strip of
                                   w = min(tile_w, 8) columns by (32 / w) *
                                   pixels_per_thread rows (strips side by side
                                   across wider tiles): 0 = automatic, else
                                   1, 2, 4 or 8 with the strip height dividing
                                   tile_h.  Results do not depend on it. */
    int32_t smem_batch;         /* Gaussians a warp stages in shared memory per
                                   batch: 0 = automatic (128), else 64, 128 or
                                   192 (used with 4 pixels per lane; other
                                   pixel counts use 128).  Results do not
                                   depend on it. */
} mvgs_config;

/* cfg->flags bit for the sampled calls: blend whole strips and leave the
 * lanes of unsampled pixels idle (the naive partial rendering of Fig. 3b),
 * instead of packing the samples into runs (Alg. 3).  Same results; for
 * comparison. */
#define MVGS_FLAG_MASKED_PARTIAL 1u
/* cfg->flags bit for the forward calls: also write each rendered pixel's
 * expected depth sum_i alpha_i T_i z_i (z_i the camera depth of the i-th
 * blended Gaussian; not divided by the accumulated opacity) into the state
 * array at layout.off_pixel_depth, for the 3D distance-aware D-SSIM. */
#define MVGS_FLAG_DEPTH 2u
/* cfg->flags bit for the forward calls: capturable mode.  The record and key
 * counts are not read back; every launch is sized by `cap` and stops at the
 * counts held in device memory, so the call never synchronises and can be
 * captured in a CUDA graph (with the backward, the losses and the ADC call).
 * `needed` gets -1s.  Results are valid only if the counts block of the state
 * (layout.off_counts) shows needed counts within the capacity afterwards:
 * otherwise the records and keys past it were dropped, and the caller grows
 * the buffers and runs again. */
#define MVGS_FLAG_CAPTURABLE 4u
/* cfg->flags bit for the forward calls: also write the per-pixel statistics
 * (layout.off_pixel_stats: where the pixel stopped and how many Gaussians it
 * blended).  Counting costs about 5% of the blend forward, so it is off by
 * default and the array is then left as it was. */
#define MVGS_FLAG_PIXEL_STATS 8u

/* Capacities the caller sized `state` and `workspace` for:
 * records = visible (Gaussian, view) pairs, keys = (record, tile) pairs. */
typedef struct mvgs_capacity {
    int64_t records;
    int64_t keys;
} mvgs_capacity;

/* Byte offsets of the arrays inside `state` (all 256-byte aligned), so a
 * caller may read the intermediate results, and the total sizes. */
typedef struct mvgs_layout {
    size_t state_bytes;
    size_t workspace_bytes;          /* forward and backward scratch (max of both) */
    size_t off_counts;               /* int64[6]: records and keys held, tiles, pixels,
                                        records and keys the batch needed          */
    size_t off_rec_offsets;          /* int64[n + 1]: records of Gaussian g are
                                        [off[g], off[g+1]) (Gaussian-major)       */
    size_t off_rec_gauss;            /* int32[records]: Gaussian index            */
    size_t off_rec_view;             /* int32[records]: view index                */
    size_t off_rec_xy;               /* float2[records]: projected mean (pixels)   */
    size_t off_rec_conic_opacity;    /* float4[records]: conic A, B, C; opacity   */
    size_t off_rec_rgb;              /* float4[records]: rgb; .w = radius in pixels */
    size_t off_rec_clamp;            /* int32[records]: bit c set if channel c was
                                        clamped at 0                              */
    size_t off_rec_depth;            /* float[records]: camera depth              */
    size_t off_rec_rect;             /* int16x4[records]: tile x0, y0, x1, y1 (excl.) */
    size_t off_sorted_records;       /* uint32[keys]: record ids sorted by (view, tile, depth, Gaussian) */
    size_t off_tile_ranges;          /* int64x2[tiles]: [start, end) into the sorted ids */
    size_t off_tile_order;           /* uint32[tiles]: blend processing order (longest lists first) */
    size_t off_final_T;              /* float[pixels]: transmittance after blending */
    size_t off_n_contrib;            /* uint32[pixels]: list position one past the last contributor */
    size_t off_pixel_stats;          /* uint32x2[pixels]: list entries the pixel examined before it
                                        stopped, and the number of Gaussians it blended
                                        (with MVGS_FLAG_PIXEL_STATS) */
    size_t off_pixel_depth;          /* float[pixels]: expected depth (with MVGS_FLAG_DEPTH) */
    int64_t tiles;                   /* total tiles over all views                 */
    int64_t pixels;                  /* total pixels over all views                */
} mvgs_layout;

/* Fills `out` for a scene of n Gaussians, V host cameras and the capacities.
 * Pure host arithmetic.  Returns MVGS_EINVAL / MVGS_EOVERFLOW on bad input. */
mvgs_status mvgs_render_layout(int64_t n, const mvgs_camera* cams, int32_t V, const mvgs_config* cfg,
                               const mvgs_capacity* cap, mvgs_layout* out);

/* Participation pre-count (the supplement's test of which Gaussians take part
 * in which view, done before anything is allocated): the exact record and key
 * counts mvgs_render_views will need for this scene, cameras and tile size,
 * without writing records.  For admission and for sizing buffers (e.g. a
 * capturable rasterizer) ahead of a batch.  Synchronises `stream`. */
size_t mvgs_count_workspace_size(int64_t n, int32_t V);
mvgs_status mvgs_count_views(const mvgs_scene* scene, const mvgs_camera* cams, int32_t V, const mvgs_config* cfg,
                             mvgs_capacity* needed, void* workspace, size_t workspace_bytes, mvgs_stream stream);

/* Forward render of V views (Eq. 1; preprocessing of the supplement).
 *   images     [3 * pixels] float32 out, packed per view (see top).
 *   state      >= layout.state_bytes, written; keep it for the backward.
 *   workspace  >= layout.workspace_bytes, scratch.
 *   needed     out (host): the record and key counts this batch needs.
 * If a count exceeds `cap`, returns MVGS_ENOSPACE after reporting `needed`;
 * the caller re-sizes with mvgs_render_layout and calls again.
 * Synchronises `stream` twice (record and key count read-back). */
mvgs_status mvgs_render_views(const mvgs_scene* scene, const mvgs_camera* cams, int32_t V, const mvgs_config* cfg,
                              const mvgs_capacity* cap, float* images, void* state, size_t state_bytes,
                              void* workspace, size_t workspace_bytes, mvgs_capacity* needed, mvgs_stream stream);

/* Backward of mvgs_render_views for the same scene, cameras, config and
 * capacity, given dL/dimages (packed like the images).  Overwrites
 *   g_means [n,3], g_log_scales [n,3], g_quats [n,4] (w.r.t. the raw
 *   quaternion), g_opacity_logits [n], g_sh [n,(d+1)^2,3]
 * with gradients summed over all views.  Optional per-record outputs (NULL
 * to skip), indexed like the state's record arrays:
 *   g_mean2d [records, 2]  dL/d projected mean, pixel units;
 *   e1       [records]     sum over pixels of the norm of each pixel's
 *                          contribution to dL/d projected mean.
 * `state` is read-only. */
mvgs_status mvgs_render_views_backward(const mvgs_scene* scene, const mvgs_camera* cams, int32_t V,
                                       const mvgs_config* cfg, const mvgs_capacity* cap, const float* dL_dimages,
                                       const void* state, size_t state_bytes, void* workspace,
                                       size_t workspace_bytes, float* g_means, float* g_log_scales, float* g_quats,
                                       float* g_opacity_logits, float* g_sh, float* g_mean2d, float* e1,
                                       mvgs_stream stream);

/* ---- thread-efficient partial rendering (Sec. 5.1.1, Alg. 3, Fig. 3c) ----
 * Each (view, tile) renders only a sub-sample of its pixels, given as an
 * index array per (tile, view): the blend packs the samples of a tile into
 * runs of 32 * pixels_per_thread, one warp each, so no lane idles on an
 * unsampled pixel.  The sort and the tile lists are those of the full render.
 *
 * A sample set, device arrays owned by the caller:
 *   offsets [layout.tiles + 1] int64: the samples of global tile t (view-major
 *           tile numbering, row-major tiles inside a view) are
 *           pixels[offsets[t] .. offsets[t + 1]);
 *   pixels  uint16 pixel index inside the tile, ly * tile_w + lx, at most
 *           layout.pixels entries in all.  Indices outside the image or the
 *           tile are skipped; a pixel listed twice is rendered twice. */
typedef struct mvgs_samples {
    const int64_t* offsets;
    const uint16_t* pixels;
} mvgs_samples;

/* The sampling rule: group, cell size and seed (see mvgs_partial_samples). */
typedef struct mvgs_sampling {
    int32_t group;          /* views sharing the pixel positions of a tile */
    int32_t cell_w, cell_h; /* pixels decided together (1 x 1: pixel by pixel) */
    uint64_t seed;
} mvgs_sampling;

/* Scratch bytes for mvgs_partial_samples. */
size_t mvgs_partial_samples_workspace_size(const mvgs_camera* cams, int32_t V, const mvgs_config* cfg);

/* Fills a sample set: view v renders pixel (x, y) when its cell
 * (cx, cy) = (x / cell_w, y / cell_h) has
 *   floor(group * (h >> 32) / 2^32) == v mod group,
 * h = SplitMix64 output number 2^32 cy + cx + 1 of the stream seeded with
 * `seed`.  So `group` consecutive views of one resolution split every pixel
 * position between them exactly once (one image's worth of pixels over
 * `group` views), each taking about 1/group of its pixels.  The paper leaves
 * the sub-sampling rule open; this one is seeded and reproducible.  Cells of
 * tile_w x (32 / tile_w) * pixels_per_thread pixels are exactly the warps'
 * strips, which keeps every run of samples compact (best culling).
 *   offsets [layout.tiles + 1], pixels [layout.pixels]: device, written.
 * The tile size in cfg must be the one used to render. */
mvgs_status mvgs_partial_samples(const mvgs_camera* cams, int32_t V, const mvgs_config* cfg,
                                 const mvgs_sampling* sampling, int64_t* offsets, uint16_t* pixels, void* workspace,
                                 size_t workspace_bytes, mvgs_stream stream);

/* mvgs_render_views restricted to a sample set: writes the images,
 * final_T, n_contrib (and with the flags the depth and pixel statistics) of
 * the sampled pixels only (every other pixel of `images` and of those state
 * arrays is left as it was).  A sampled pixel gets exactly the value the full
 * render gives it. */
mvgs_status mvgs_render_views_sampled(const mvgs_scene* scene, const mvgs_camera* cams, int32_t V,
                                      const mvgs_config* cfg, const mvgs_capacity* cap, const mvgs_samples* samples,
                                      float* images, void* state, size_t state_bytes, void* workspace,
                                      size_t workspace_bytes, mvgs_capacity* needed, mvgs_stream stream);

/* Backward of mvgs_render_views_sampled (same sample set): only the sampled
 * pixels of dL_dimages are read; equals the full backward with dL_dimages
 * zero at every unsampled pixel. */
mvgs_status mvgs_render_views_sampled_backward(const mvgs_scene* scene, const mvgs_camera* cams, int32_t V,
                                               const mvgs_config* cfg, const mvgs_capacity* cap,
                                               const mvgs_samples* samples, const float* dL_dimages,
                                               const void* state, size_t state_bytes, void* workspace,
                                               size_t workspace_bytes, float* g_means, float* g_log_scales,
                                               float* g_quats, float* g_opacity_logits, float* g_sh,
                                               float* g_mean2d, float* e1, mvgs_stream stream);

/* ---- 3D distance-aware D-SSIM (Sec. 5.1.2) on merged images (Fig. 3c) ----
 * A partially rendered batch puts, at every pixel position, the pixel of one
 * view of its group into the "merged" image; neighbours there may come from
 * different viewpoints, so SSIM's window is replaced by a kernel on 3D
 * distances between the pixels' surface points.  Views are taken in groups
 * of `group` consecutive views of one resolution (V a multiple of group);
 * merged image m (packed like the images: [3, H, W] after the previous
 * merged images) takes pixel (x, y) from view m * group + slot(x, y), the
 * view that rendered it under mvgs_partial_samples with the same sampling
 * rule. */

/* Scratch bytes of mvgs_merge_views / mvgs_split_merged_grad. */
size_t mvgs_merge_workspace_size(int32_t V);

/* Builds the merged images.  Inputs (device, packed per view): images and
 * targets [3 * pixels], and depth_acc and final_T [pixels] from a forward run
 * with MVGS_FLAG_DEPTH (the state arrays at layout.off_pixel_depth and
 * off_final_T).  Outputs (device, packed per merged image; any may be NULL
 * to skip, points and sigma together):
 *   merged_img, merged_tgt [3, H, W]  the owner view's colour / target;
 *   points [3, H, W]  surface point X = R^T (z K^-1 (x + 0.5, y + 0.5, 1) - t)
 *                     of the owner view, z = depth_acc / (1 - final_T);
 *   sigma  [H, W]     kernel width sigma_px * z / f_x (sigma_px: the 2D
 *                     window's sigma, 1.5), 0 where 1 - final_T < 1e-3 (no
 *                     surface point; such a pixel is only its own neighbour). */
mvgs_status mvgs_merge_views(const mvgs_camera* cams, int32_t V, const mvgs_sampling* sampling, float sigma_px,
                             const float* images, const float* targets, const float* depth_acc, const float* final_T,
                             float* merged_img, float* merged_tgt, float* points, float* sigma, void* workspace,
                             size_t workspace_bytes, mvgs_stream stream);

/* Sends dL/d(merged images) back to the views: each view pixel gets the
 * merged gradient where it is the owner and 0 elsewhere (dL_dimages is
 * fully written, packed per view). */
mvgs_status mvgs_split_merged_grad(const mvgs_camera* cams, int32_t V, const mvgs_sampling* sampling,
                                   const float* dL_dmerged, float* dL_dimages, void* workspace,
                                   size_t workspace_bytes, mvgs_stream stream);

/* Scratch bytes of mvgs_dssim3d_loss for M images (hw: host [M, 2]). */
size_t mvgs_dssim3d_workspace_size(const int32_t* hw, int32_t M);

/* Per-image L_m = (1 - lambda) mean|I - I*| + lambda (1 - mean SSIM*), SSIM*
 * with K*(p, q) = exp(-|X_q - X_p|^2 / (2 s_p^2)) over the 11x11 pixel
 * window of p, normalised to sum 1 over the neighbours inside the image with
 * s > 0 (p itself always counts), C1 = 0.01^2, C2 = 0.03^2; means over the
 * 3 channels and all pixels.
 *   img, target, points [3, H, W] and sigma [H, W] per image, packed;
 *   loss_per_image [M] out; dL_dimg (packed, or NULL) out: d(mean_m L_m)/d img
 *   with the kernel weights held constant.  Deterministic. */
mvgs_status mvgs_dssim3d_loss(const float* img, const float* target, const float* points, const float* sigma,
                              const int32_t* hw, int32_t M, float lambda, float* loss_per_image, float* dL_dimg,
                              void* workspace, size_t workspace_bytes, mvgs_stream stream);

/* ---- training-loop pieces: multi-view densification (Sec. 5.2.2) and Adam ----
 * Thresholds in the parameters' own spaces; decisions per Gaussian, taken in
 * double precision from the float32 inputs:
 *   mean E_k = accum_E_k / denom (0 where denom = 0);
 *   large    = max_i log_scale_i > log_dense_extent;
 *   pruned   = opacity_logit < prune_logit (the supplement multiplies the
 *              opacity threshold by the views per iteration);
 *   split    = !pruned && large && mean E_1 >= split_threshold;
 *   cloned   = !pruned && !large && mean E_2 >= clone_threshold
 *   (E_1 is good at splitting and E_2 at cloning, Sec. 5.2.2). */
typedef struct mvgs_densify_params {
    double split_threshold;
    double clone_threshold;
    double prune_logit;
    double log_dense_extent;
} mvgs_densify_params;

size_t mvgs_densify_workspace_size(int64_t n);

/* One densification step.  Outputs, ordered by source Gaussian: none for a
 * pruned Gaussian; for a split one two children with mean mu + R(q)(s * z_k)
 * (z = normals [n, 2, 3], the caller's standard normal samples), log-scale
 * reduced by ln 1.6 and the rest copied; for a cloned one the Gaussian and a
 * copy; else the Gaussian.  out_* are device arrays of `capacity` Gaussians
 * (same layouts as the scene); out_src [capacity] int64 source index and
 * out_kind [capacity] int32 (0 the Gaussian itself, 1 a clone's copy, 2 a
 * split child) may be NULL.  Synchronises the stream once to read the output
 * count into *n_out; if it exceeds `capacity`, returns MVGS_ENOSPACE (with
 * *n_out set) and writes nothing. */
mvgs_status mvgs_densify(const mvgs_scene* scene, const float* accum_e1, const float* accum_e2, const float* denom,
                         const float* normals, const mvgs_densify_params* params, int64_t capacity,
                         float* out_means, float* out_log_scales, float* out_quats, float* out_opacity_logits,
                         float* out_sh, int64_t* out_src, int32_t* out_kind, int64_t* n_out, void* workspace,
                         size_t workspace_bytes, mvgs_stream stream);

/* Carries a per-Gaussian array (`width` floats each, e.g. optimiser moments)
 * through a densification step: out[d] = in[src[d]] where kind[d] == 0, else
 * zeros. */
mvgs_status mvgs_densify_carry(int64_t n_out, const int64_t* src, const int32_t* kind, int32_t width,
                               const float* in, float* out, mvgs_stream stream);

/* Adam (Kingma & Ba 2015) with bias correction on `count` floats in place:
 * m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2;
 * p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).  step >= 1. */
mvgs_status mvgs_adam_step(int64_t count, float* param, const float* grad, float* m, float* v, float lr, float beta1,
                           float beta2, float eps, int32_t step, mvgs_stream stream);

/* Scratch bytes mvgs_dssim_loss needs for these views (hw: host [V, 2] of
 * (height, width)). */
size_t mvgs_dssim_workspace_size(const int32_t* hw, int32_t V);

/* Per-view loss L_v = (1 - lambda) mean|I - I*| + lambda (1 - SSIM(I, I*)),
 * SSIM with an 11x11 Gaussian window (sigma 1.5, normalised to sum 1), zero
 * padding, C1 = 0.01^2, C2 = 0.03^2, averaged over the 3 channels and all
 * pixels of the view.
 *   img, target  packed images (see top)   loss_per_view [V] float32 out
 *   dL_dimg      packed, out: d(mean_v L_v)/d img; NULL to skip.
 * Deterministic (no atomics). */
mvgs_status mvgs_dssim_loss(const float* img, const float* target, const int32_t* hw, int32_t V, float lambda,
                            float* loss_per_view, float* dL_dimg, void* workspace, size_t workspace_bytes,
                            mvgs_stream stream);

/* mvgs_dssim_loss without a caller workspace, for callers that cannot
 * allocate device memory (a plug-in inside another framework's memory pool, a
 * process that reserves all device memory up front, a loop that must never
 * enter the allocator).  No counterpart in the paper.  Same arguments and
 * results as mvgs_dssim_loss minus the workspace: the scratch is an 80 MiB
 * static device array inside the library (every GPU that loads the library
 * holds it until exit), enough for about 2.2 million pixels per call (one
 * 1920x1080 view); larger calls return MVGS_ENOSPACE without launching.  Each
 * call outside stream capture looks up the array's address on the current
 * device and caches it; a call under capture uses the cached address, so make
 * a device's first call before any capture (a first call under capture returns
 * MVGS_ECUDA without launching).  Calls share the array, so calls that overlap
 * on the GPU race; nothing in it needs clearing between calls.  Timed as the
 * D-SSIM stage when stage timing is on. */
mvgs_status mvgs_dssim_loss_noalloc(const float* img, const float* target, const int32_t* hw, int32_t V,
                                    float lambda, float* loss_per_view, float* dL_dimg, mvgs_stream stream);

/* Adds this batch's densification statistics into running per-Gaussian sums
 * (Sec. 5.2.2):
 *   accum_e1[g] += sum_views e1[record]           (E_1: norm, then add)
 *   accum_e2[g] += sum_views || g_mean2d[record] || (E_2: add per view, norm)
 *   denom[g]    += number of views in which g is visible
 * `state` is the forward's state for the batch (its record map is read);
 * g_mean2d / e1 are the per-record outputs of the backward. */
mvgs_status mvgs_adc_accumulate(const void* state, int64_t n, const float* g_mean2d, const float* e1,
                                float* accum_e1, float* accum_e2, float* denom, mvgs_stream stream);

/* Optional stage timing (instrumentation; the paper has no counterpart).
 * While enabled, every call records a pair of CUDA events around each of its
 * stages on the call's stream (events are host objects; no device memory is
 * allocated).  mvgs_profile_read waits for the recorded events, adds their
 * durations to per-stage totals, copies up to max_stages totals (ms) and
 * launch counts into the host arrays, resets them, and returns the number of
 * stages.  Process-wide; intended for one calling thread at a time. */
typedef enum mvgs_stage {
    MVGS_STAGE_COUNT_VISIBLE = 0, /* participation count per (Gaussian, view)  */
    MVGS_STAGE_SCAN_RECORDS,      /* record offsets                            */
    MVGS_STAGE_PREPROCESS,        /* projection, colour, radius, rect          */
    MVGS_STAGE_DEPTH_SORT,        /* records by depth                          */
    MVGS_STAGE_SCAN_TILES,        /* key offsets                               */
    MVGS_STAGE_TILE_SORT,         /* one entry per (record, tile), generated
                                     in the first pass, sorted by (view, tile) */
    MVGS_STAGE_RANGES,            /* per-tile list ranges from the rectangles  */
    MVGS_STAGE_BLEND_FORWARD,
    MVGS_STAGE_ZERO_GRADS,
    MVGS_STAGE_BLEND_BACKWARD,
    MVGS_STAGE_PREPROCESS_BACKWARD,
    MVGS_STAGE_DSSIM,
    MVGS_STAGE_ADC,
    MVGS_STAGE_COUNT
} mvgs_stage;
mvgs_status mvgs_profile_enable(int32_t on);
int32_t mvgs_profile_read(float* total_ms, int64_t* launches, int32_t max_stages);
const char* mvgs_stage_name(int32_t stage);

/* Number of CUDA kernels the library has launched in this process (all
 * threads and streams), for accounting in benchmarks. */
int64_t mvgs_launch_count(void);

/* Message of the last failed call on this thread ("" if none). */
const char* mvgs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MVGS_H */
