/*
 * pbr.h -- C ABI of libpbr.so, the GB300 (sm_103a) point-splat renderer.
 *
 * The renderer implements the differentiable splatting of Zhang et al.,
 * "Differentiable Point-Based Radiance Fields for Efficient View Synthesis"
 * (SIGGRAPH Asia 2022):
 *   Sec. 3.1, Eq. 1    projection p = (M (R P + t))v of every point;
 *   Sec. 3.1, Eqs. 2-4 per-point SH colour c = sum_lm h_lm Y_lm(v), with the
 *                      view direction v = (R P + t)/|R P + t| (Eq. 3);
 *   Sec. 3.2, Eq. 5    image-space Gaussian kernel per point and pixel;
 *   Sec. 3.2, Eqs. 6-7 depth sort and front-to-back alpha blending, limited
 *                      to points within a cutoff distance of the pixel;
 *   Sec. 3.3           gradients of the image w.r.t. positions and SH
 *                      coefficients for end-to-end training, the Eq. 8
 *                      objective and optimiser step, and the hybrid
 *                      coarse-to-fine point update (Algorithm 1);
 *   Sec. 3.4           video frame initialisation (Chamfer descent and
 *                      parameter transfer);
 *   Sec. 3.1, appendix visual-hull initialisation and consistency check.
 *
 * Conventions shared by every entry point
 *   - Every function returns an int status: PBR_OK (0) or a negative
 *     PBR_ERR_* code; pbr_last_error(ctx) returns a message for the calling
 *     thread.  No C++ exception crosses this boundary.
 *   - Point arrays, images and gradient buffers are DEVICE pointers owned by
 *     the caller (fp32, C-contiguous); cameras and options are HOST structs.
 *     The caller keeps the point arrays alive and unchanged between a forward
 *     call and the backward call that uses its state.
 *   - The library owns the context, the forward state, graphs and resident
 *     scenes; each has a matching destroy/free call.
 *   - Work is enqueued on the given cudaStream_t (NULL = legacy default
 *     stream).  Calls return when the work is enqueued, except where a
 *     comment says the call synchronises.
 *   - Images are packed per view in view order: view v occupies
 *     [pix_base(v), pix_base(v) + H_v W_v) pixels of 3 floats (RGB),
 *     row-major, pixel (0,0) at the top-left.
 *
 * Camera model (Sec. 3.1): X = R P + t (R row-major, world -> camera), the
 * camera looks down +z, x right, y down; pixel centres at (x+0.5, y+0.5);
 * p = (fx X.x/X.z + cx, fy X.y/X.z + cy).
 */
#ifndef PBR_H
#define PBR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *pbr_stream_t; /* same type as cudaStream_t */

enum {
    PBR_OK = 0,
    PBR_ERR_INVALID_ARG = -1,
    PBR_ERR_OOM = -2,
    PBR_ERR_CUDA = -3,
    PBR_ERR_CAPACITY = -4,
    PBR_ERR_TIMEOUT = -5,
    PBR_ERR_DEVICE_STATUS = -6,
    PBR_ERR_NOT_FOUND = -7,
    PBR_ERR_BUSY = -8
};

typedef struct pbr_ctx pbr_ctx;
typedef struct pbr_state pbr_state;
typedef struct pbr_graph pbr_graph;

/* One pinhole camera (Sec. 3.1, Eq. 1: intrinsics M = (fx, fy, cx, cy),
 * extrinsics (R, t)) and the size of the image it renders. */
typedef struct {
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    int32_t width, height;
} pbr_camera;

/* Renderer options.  pbr_default_opts() fills the defaults listed here. */
typedef struct {
    int32_t radius_mode;   /* 0 (default): kernel width s = fx * r / z pixels;
                              1: s = r * min(W, H) / 2 (fixed image-space radius) */
    int32_t dir_frame;     /* 0 (default): SH direction in the camera frame as in
                              Sec. 3.1 Eq. 3; 1: world-frame direction R^T v */
    float cutoff_k;        /* cutoff radius = cutoff_k * s (default 3) */
    float alpha_max;       /* alpha = min(alpha_max, o * G), default 0.99, < 1 */
    float t_eps;           /* stop once transmittance < t_eps (default 1e-5); values
                              below 1e-30 act as 1e-30 (T stays a normal fp32 number
                              for the backward's recovery of T) */
    int32_t max_per_pixel; /* composite at most this many points (0 = no cap) */
    float bg[3];           /* background colour (default 0) */
    float z_near;          /* points with z <= z_near are culled (default 0.01) */
    int32_t tile_w, tile_h;/* tile size: 8x8, 16x16 (default) or 16x32 */
    int32_t batch_depth;   /* compositing schedule: 0 (default) = warp-streamed (each
                              warp walks its tile list alone, no block barriers);
                              32..1024 (multiple of 32) = block-staged batches of
                              that many points in shared memory */
    int32_t persistent;    /* 1: warp-streamed compositing as one persistent launch
                              (SM-count grid, warps pull (tile, 8x8 sub-block)
                              items longest tile first); 0 (default): one block
                              per tile.  Ignored by the block-staged schedule. */
    int32_t no_pair_stats; /* 1: the compositing kernels skip the pair counting
                              that pbr_state_stats reports (as captured graphs
                              always do); 0 (default): count */
    int32_t bwd_mode;      /* how the backward pass gets the transmittance T each
                              pixel had before each composited point (Sec. 3.3
                              end-to-end gradients need it):
                              1 recompute: from T after the last point, dividing
                                by (1 - alpha) back to front (no memory beyond
                                T_final and the list position per pixel);
                              2 store: the forward keeps T before each of the
                                first store_depth composited points of every
                                pixel (4 store_depth + 4 bytes per pixel; deeper
                                points fall back to recomputation);
                              0 auto (default): store when that list takes at
                                most an eighth of the context's HBM budget, else
                                recompute.  The block-staged schedule and
                                captured graphs always recompute.
                              Store mode keeps T exact (no division); it is
                              not faster: writing and reading the list costs
                              more than the reciprocal and multiply per
                              composited point it saves (on the 1M-point,
                              64-view step, 34.0 against 24.3 ms), so callers
                              after speed set 1. */
    int32_t store_depth;   /* composited points per pixel whose T is kept in store
                              mode (0 = default 32; at most 255) */
} pbr_render_opts;

/* One scene: n points with position [n,3], SH coefficients [n,K,3]
 * (K = (sh_degree+1)^2, coefficient k = l*l + l + m, RGB innermost),
 * kernel amplitude (opacity) [n] and radius [n].  Device pointers. */
typedef struct {
    const float *pos;
    const float *sh;
    const float *opacity;
    const float *radius;
    int64_t n;
    int32_t sh_degree; /* 0..3 */
    int32_t reserved;
} pbr_points;

/* Sizes of one forward pass (filled by pbr_state_info). */
typedef struct {
    int64_t n_point_views; /* sum over views of the scene's point count */
    int64_t n_visible;     /* point-views that survive culling */
    int64_t n_pairs;       /* (tile, point-view) pairs after binning */
    int64_t n_tiles;       /* tiles over all views */
    int64_t n_pixels;      /* pixels over all views */
    /* device pointers into the state (valid until pbr_state_free) */
    const uint32_t *tile_keys;  /* [n_pairs] sorted keys: global tile id << B | block mask,
                                   B = (tile_w / 8) (tile_h / 8) when that exceeds 1, else 0;
                                   bit by (tile_w / 8) + bx of the mask is set iff a pixel of
                                   the tile's 8 x 8 block (bx, by) passes the point-view's
                                   cutoff test.  A tile lists a point-view iff one of its
                                   pixels does (Sec. 3.2 cutoff). */
    const uint32_t *tile_vals;  /* [n_pairs] point-view id, (tile, depth, id) order */
    const uint32_t *ranges;     /* [n_tiles][2] start, end into the lists */
    const float *records;       /* [n_point_views][8] px, py, rc^2, q', o, r, g, b */
    const uint32_t *ntiles;     /* [n_point_views] tiles covered (0 = culled) */
    const float *T_final;       /* [n_pixels] transmittance after compositing */
    const uint32_t *n_contrib;  /* [n_pixels] list position after the last composited point */
} pbr_state_info_t;

/* ---------------------------------------------------------------- context */
/* Creates a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * memory the serving loop may hold for in-flight requests (0 = 80% of free
 * device memory at creation). */
int pbr_create(pbr_ctx **out, int device, size_t hbm_budget_bytes);
int pbr_destroy(pbr_ctx *ctx);
/* Message for the last error of a pbr_* call on the calling thread ("" if
 * none).  The message is kept per thread, not per context: ctx may be NULL
 * (e.g. after a failed pbr_create) and is not dereferenced. */
const char *pbr_last_error(const pbr_ctx *ctx);
void pbr_default_opts(pbr_render_opts *opts);
/* Library version string and the compiled SM architecture. */
const char *pbr_version(void);

/* ---------------------------------------------------------------- render */
/* Forward pass (Sec. 3.1 Eqs. 1-4, Sec. 3.2 Eqs. 5-7) of n_cams views in
 * one batch.  Views may belong to different scenes: scene_of_view[v] (host
 * array, NULL = all views of scene 0) picks scenes[]; a multi-frame video is
 * n_scenes = frames.  out_rgb: device [sum_v H_v W_v, 3] fp32.
 * state_out: when non-NULL receives the state the backward pass needs (owned
 * by the library; free with pbr_state_free); when NULL the pass is
 * forward-only and keeps nothing.  Synchronises the stream once (to size the
 * tile lists).  Errors: INVALID_ARG (bad sizes, degree, options), OOM,
 * CUDA, DEVICE_STATUS (a kernel flagged an inconsistent count). */
int pbr_render_forward(pbr_ctx *ctx, const pbr_points *scenes, int32_t n_scenes,
                       const int32_t *scene_of_view, const pbr_camera *cams, int32_t n_cams,
                       const pbr_render_opts *opts, float *out_rgb, pbr_state **state_out,
                       pbr_stream_t stream);

/* Device memory a pbr_render_forward call with these arguments would
 * allocate, at its peak (the forward state and the call's temporaries), so
 * that a caller (or the serving loop's admission) can plan by memory.  Runs
 * the per-point stage once, counting only (it writes no per-point record), to
 * learn the number of visible point-views and (tile, point-view) pairs of
 * Sec. 3.2's binning, and synchronises the stream.
 *   keep_state : 1 = the caller will ask for the state (state_out non-NULL),
 *                which adds the stored transmittance list when opts->bwd_mode
 *                resolves to store; 0 = a forward-only call.
 *   bytes      : receives the peak bytes.
 *   store_bytes: (nullable) receives the bytes of the stored transmittance
 *                list alone (0 when the mode resolves to recompute).
 * Errors as pbr_render_forward. */
int pbr_forward_workspace_size(pbr_ctx *ctx, const pbr_points *scenes, int32_t n_scenes,
                               const int32_t *scene_of_view, const pbr_camera *cams,
                               int32_t n_cams, const pbr_render_opts *opts, int32_t keep_state,
                               size_t *bytes, size_t *store_bytes, pbr_stream_t stream);

/* Backward pass (Sec. 3.3) for L with dL/dI = grad_rgb (device, packed like
 * out_rgb).  Gradients are OVERWRITTEN, packed over scenes in scene order:
 * grad_pos [sum_s n_s, 3], grad_sh [sum_s n_s K_s 3], grad_opacity [sum_s n_s]
 * (nullable); the slices of scenes that no view sees are set to zero.  Does
 * not synchronise. */
int pbr_render_backward(pbr_ctx *ctx, pbr_state *state, const float *grad_rgb, float *grad_pos,
                        float *grad_sh, float *grad_opacity, pbr_stream_t stream);
int pbr_state_free(pbr_ctx *ctx, pbr_state *state);
/* Sizes and device pointers of a forward state (for inspection and tests).
 * Synchronises the state's stream. */
int pbr_state_info(pbr_state *state, pbr_state_info_t *info);

/* Copies one array of a forward state into host memory (inspection and
 * tests).  which: 0 tile keys (as in pbr_state_info_t), 1 tile values
 * (point-view ids), 2 ranges, 3 records, 4 tile counts, 5 T_final,
 * 6 n_contrib, 7 the stored transmittances (store mode: [n_pixels][store_depth]
 * fp32, T before the k-th composited point of each pixel), 8 the number of
 * points composited per pixel (store mode, u32).  Copies
 * min(cap_bytes, size) bytes; *size_bytes receives the full size.
 * Synchronises the state's stream. */
int pbr_state_read(pbr_state *state, int32_t which, void *host_dst, size_t cap_bytes,
                   size_t *size_bytes);

/* Image loss used by the training step: kind 0 = sum of squared errors
 * (Sec. 3.3 Eq. 8, data term), kind 1 = sum of absolute errors.  Writes
 * dL/dpred into grad (device, n floats) and adds the loss to *loss_dev
 * (device double, caller zeroes it). */
int pbr_image_loss(int32_t kind, const float *pred, const float *target, int64_t n, float *grad,
                   double *loss_dev, pbr_stream_t stream);

/* Raster pair counts of a forward state (and of the backward passes run on
 * it): out4 = {forward pairs examined, forward pairs composited, backward
 * pairs examined, backward pairs contributing}.  Composited and contributing
 * pairs are the work units of the compositing kernels' ALU roofline; the
 * examined counts depend on the schedule's culling.  Only eager passes
 * (pbr_render_forward / pbr_render_backward) without opts.no_pair_stats
 * count; captured graphs (pbr_graph_*) run kernels without the counting.
 * Synchronises the state's stream. */
int pbr_state_stats(pbr_state *state, unsigned long long *out4);

/* ------------------------------------------------------- batched graphs */
/* Plans one batch of views (the same arguments as pbr_render_forward) and
 * captures it as CUDA graphs that replay without any host synchronisation:
 * an eager planning pass measures the pair count and depth range, buffers
 * are allocated once (pairs x (1 + headroom)), and the forward chain -- and,
 * when gradient buffers are given, the backward pass and a whole training
 * step (forward, image loss against `target`, backward) -- are captured.
 * Graph phases for pbr_graph_launch: 0 forward (writes out_rgb), 1 backward
 * (reads grad_rgb; with grad_rgb NULL and a target, the dL/dI that the last
 * phase 2 or 3 replay wrote), 2 forward + loss + backward
 * (needs target; writes the loss to loss_out when non-NULL and gradients to
 * grad_*), 3 full training iteration (after pbr_graph_set_optimizer).
 * The point arrays and output buffers are bound at capture: update their
 * contents in place between launches (e.g. after an optimiser step).
 * loss_kind: 0 sum of squares, 1 sum of absolute values.  Synchronises the
 * stream during planning.  Errors: INVALID_ARG, OOM, CUDA. */
int pbr_graph_create(pbr_ctx *ctx, const pbr_points *scenes, int32_t n_scenes,
                     const int32_t *scene_of_view, const pbr_camera *cams, int32_t n_cams,
                     const pbr_render_opts *opts, float *out_rgb, const float *target,
                     int32_t loss_kind, double *loss_out, const float *grad_rgb, float *grad_pos,
                     float *grad_sh, float *grad_opacity, double headroom, pbr_stream_t stream,
                     pbr_graph **out);
/* Enqueues one replay of a phase on `stream`. */
int pbr_graph_launch(pbr_graph *graph, int32_t phase, pbr_stream_t stream);
/* Synchronises `stream` and reads the device status word: PBR_ERR_CAPACITY
 * when the last replay had more pairs than planned or depths outside the
 * planned key range (its output is then invalid: call pbr_graph_replan and
 * launch again).  Optional outputs: pair count of the last replay and the
 * planned capacity. */
int pbr_graph_check(pbr_graph *graph, pbr_stream_t stream, int64_t *n_pairs, int64_t *cap_pairs);
/* Re-plans on the current point data and re-captures (synchronises). */
int pbr_graph_replan(pbr_graph *graph, pbr_stream_t stream);
/* Replaces the cameras' intrinsics and extrinsics (image sizes must be
 * unchanged) for the following launches.  Synchronises the stream. */
int pbr_graph_set_cameras(pbr_graph *graph, const pbr_camera *cams, int32_t n_cams,
                          pbr_stream_t stream);
int pbr_graph_destroy(pbr_graph *graph);

/* Autotuner: times every schedule candidate (tile 8x8 / 16x16 / 16x32 x
 * {warp-streamed, persistent warp-streamed, block-staged 128 / 256 / 512})
 * on this batch -- forward only (mode 0) or forward + backward (mode 1),
 * `reps` timed runs each -- and writes the fastest into *opts (tile_w,
 * tile_h, batch_depth, persistent).  The choice is cached in the context
 * per shape class (views, log2 pixels, log2 point-views, SH degrees, mode);
 * a cached class returns at once unless ms_out is given.  ms_out (nullable,
 * 15 entries) receives the mean milliseconds per candidate in the order
 * above, *n_candidates the number timed.  Synchronises. */
int pbr_autotune(pbr_ctx *ctx, const pbr_points *scenes, int32_t n_scenes,
                 const int32_t *scene_of_view, const pbr_camera *cams, int32_t n_cams,
                 pbr_render_opts *opts, int32_t mode, int32_t reps, double *ms_out,
                 int32_t *n_candidates, pbr_stream_t stream);
/* The autotuner's cache on disk (host only, no device work).
 * pbr_autotune_save writes every cached shape class and its schedule to
 * `path` (UTF-8 JSON: {"format": "pbr-autotune-1", "classes": [{"views",
 * "log2_pixels", "log2_point_views", "degrees", "mode", "tile_w", "tile_h",
 * "batch_depth", "persistent"}, ...]}, integers), through a temporary file
 * renamed over `path`.  pbr_autotune_load merges such a file into the
 * context's cache (its entries replace cached ones of the same class) and
 * reports the number of entries in *n_loaded (nullable).  The file is read
 * whole and checked before the cache changes: PBR_ERR_NOT_FOUND if it
 * cannot be opened, PBR_ERR_INVALID_ARG if it is not such a file or holds
 * a schedule pbr_render_forward would reject; the cache is then unchanged.
 * Not thread-safe against a concurrent pbr_autotune on the same context. */
int pbr_autotune_save(const pbr_ctx *ctx, const char *path);
int pbr_autotune_load(pbr_ctx *ctx, const char *path, int32_t *n_loaded);

/* ---------------------------------------------------------- training step */
/* Optimiser settings of the training step (Sec. 3.3: per-group learning
 * rates 3e-3 for SH coefficients and 8e-4 for positions, decayed by 0.93 per
 * epoch by the caller through pbr_graph_set_lr; objective Eq. 8 with the
 * anisotropic TV weight lambda = 0.01).  The paper says only "stochastic
 * gradient descent"; kind selects plain SGD or Adam. */
typedef struct {
    int32_t kind;                    /* 0 SGD, 1 Adam (default) */
    float lr_pos, lr_sh, lr_opacity; /* 8e-4, 3e-3, 0 (0 = group frozen) */
    float beta1, beta2, eps;         /* Adam: 0.9, 0.999, 1e-8 */
    float lambda_tv;                 /* 0.01 */
    int32_t loss_kind;               /* 0 squared error (Eq. 8, default), 1 absolute error */
    int32_t reserved[3];
} pbr_optimizer_cfg;
void pbr_default_optimizer(pbr_optimizer_cfg *cfg);

/* Eq. 8 objective over packed views (sizes from cams): adds sum over
 * pixels and channels of (pred - target)^2 (loss_kind 0) or |pred - target|
 * (1), plus lambda_tv times the anisotropic TV of pred (l1 norm of forward
 * differences along x and y, per view, per channel), to *loss_dev (device
 * double, caller zeroes it) and writes dL/dpred to grad (sign(0) = 0). */
int pbr_image_loss_tv(const pbr_camera *cams, int32_t n_cams, const float *pred,
                      const float *target, int32_t loss_kind, float lambda_tv, float *grad,
                      double *loss_dev, pbr_stream_t stream);
/* One optimiser update of n parameters in place: SGD (kind 0,
 * p -= lr g) or Adam (kind 1, moments m, v updated in place, bias
 * correction with the 1-based step number). */
int pbr_optimizer_step(int32_t kind, float *param, const float *grad, float *m, float *v,
                       int64_t n, float lr, float beta1, float beta2, float eps, int32_t step,
                       pbr_stream_t stream);
/* Adds graph phase 3, a full training iteration: forward, the Eq. 8
 * objective against the graph's target, backward, and the optimiser update
 * of the scenes' positions, SH coefficients (and opacities if lr_opacity >
 * 0) IN PLACE.  The graph must have been created with a target and gradient
 * buffers.  Optimiser moments and the step counter live in the graph (reset
 * by this call).  Synchronises. */
int pbr_graph_set_optimizer(pbr_graph *graph, const pbr_optimizer_cfg *cfg, pbr_stream_t stream);
/* New learning rates for the following phase-3 launches (epoch decay). */
int pbr_graph_set_lr(pbr_graph *graph, float lr_pos, float lr_sh, float lr_opacity);

/* ---------------------------------------------------------------- serving */
/* Statistics of the serving loop (pbr_serve_stats). */
typedef struct {
    int64_t submitted, completed, rejected, queued, in_flight_batches, batches,
        max_batch_views;
    double mean_batch_views;
    double megapixels;  /* pixels of completed requests / 1e6 */
    double span_s;      /* first arrival to last completion */
    double p50_ms, p99_ms, mean_ms, max_ms; /* arrival -> completion latency */
    size_t hbm_in_use, hbm_budget;
} pbr_serve_stats_t;

/* Starts the context's serving thread.  Requests are rendered with `opts`
 * in batches of up to max_batch_views views (any mix of scenes and image
 * sizes), with up to n_streams batches in flight on separate streams.  A
 * batch is admitted when a stream is free and its estimated workspace fits
 * in the HBM budget (pbr_create / pbr_serve_set_budget) minus what the
 * batches in flight hold; a request that cannot fit even alone is rejected
 * with PBR_ERR_OOM.  Not in the paper: the serving form of the renderer. */
int pbr_serve_start(pbr_ctx *ctx, const pbr_render_opts *opts, int32_t max_batch_views,
                    int32_t n_streams);
/* Finishes queued and in-flight requests, stops the thread, frees scenes. */
int pbr_serve_stop(pbr_ctx *ctx);
int pbr_serve_set_budget(pbr_ctx *ctx, size_t hbm_budget_bytes);
/* Copies a scene (host or device arrays, detected by unified addressing)
 * into library-owned HBM and returns its id.  Synchronous. */
int pbr_upload_scene(pbr_ctx *ctx, const pbr_points *points, int32_t *scene_id);
/* Frees a resident scene; PBR_ERR_BUSY while requests on it are pending. */
int pbr_evict_scene(pbr_ctx *ctx, int32_t scene_id);
/* Queues a forward render of scene `scene_id` from `cam` into
 * out_rgb_device ([H, W, 3] fp32, caller-owned, untouched until the request
 * completes).  arrival_time: the request's arrival on the steady clock in
 * seconds (<= 0: now), used for latency.  Returns at once with *req_id. */
int pbr_submit_request(pbr_ctx *ctx, int32_t scene_id, const pbr_camera *cam,
                       float *out_rgb_device, double arrival_time, uint64_t *req_id);
/* *done = 1 once the request has completed (its output is then final);
 * *status is its result code.  A completed request is forgotten after the
 * call that reports it done. */
int pbr_poll(pbr_ctx *ctx, uint64_t req_id, int32_t *done, int32_t *status);
/* Waits up to timeout_ms for a request; PBR_ERR_TIMEOUT if not done. */
int pbr_wait(pbr_ctx *ctx, uint64_t req_id, int32_t timeout_ms, int32_t *status);
/* Current statistics; reset != 0 clears them afterwards. */
int pbr_serve_stats(pbr_ctx *ctx, pbr_serve_stats_t *stats, int32_t reset);
/* The serving loop's steady clock (seconds), for arrival times. */
double pbr_now(void);
/* Device intervals of the batches completed since the loop started (or the
 * last reset): batch i ran on the GPU from start_ms[i] to end_ms[i]
 * (milliseconds after the loop's start, measured with CUDA events recorded
 * on the batch's stream before its first kernel and after its last), with
 * views[i] views.  Two intervals that intersect are batches whose work was on
 * the device at the same time.  Fills min(cap, *n) entries of each non-NULL
 * array; *n receives the number recorded; reset != 0 clears them. */
int pbr_serve_trace(pbr_ctx *ctx, double *start_ms, double *end_ms, int32_t *views, int32_t cap,
                    int32_t *n, int32_t reset);

/* What a request for resident scene scene_id from cam reserves from the
 * HBM budget while it is in flight (bytes): the forward pass's allocations
 * with every point-view visible and listed in as many tiles as the scene's
 * largest splat can reach from this camera (largest radius at the nearest
 * depth of the scene's bounding box), an upper bound of what
 * pbr_forward_workspace_size reports for the same view; when that bound is
 * above 1/64 of the budget (a camera near or inside the scene), the exact
 * workspace from a counting pass on the device instead.  Errors:
 * INVALID_ARG, NOT_FOUND (no such scene). */
int pbr_serve_estimate(pbr_ctx *ctx, int32_t scene_id, const pbr_camera *cam, size_t *bytes);

/* --------------------------------------------------- measurement support */
/* Number of CUDA kernels this library has launched in this process. */
unsigned long long pbr_kernel_launches(void);
/* Switches per-stage CUDA-event timing on (enable = 1) or off for the
 * context's forward and backward calls.  Stages: 0 preprocess, 1 compact,
 * 2 depth sort, 3 emit pairs, 4 tile sort, 5 tile ranges, 6 raster forward,
 * 7 raster backward (with its zeroing), 8 preprocess backward, 9 other;
 * pbr_refine_points: 10 voxel reduction, 11 neighbour searches, 12 the rest
 * (grid, outlier filter, compaction, generation). */
int pbr_set_stage_timing(pbr_ctx *ctx, int enable);
/* Accumulated milliseconds and call counts per stage since the last query
 * (arrays of n entries); resets the accumulators.  Synchronises. */
int pbr_stage_times(pbr_ctx *ctx, double *ms, long long *calls, int n);

/* ------------------------------------------------ allocation-free forward */
/* The paper has no counterpart: this is a deployment variant of
 * pbr_render_forward (forward only, no state) for callers that cannot
 * allocate device memory -- e.g. plug-ins running under a host
 * application's allocator, or real-time loops that must not call the
 * allocator after start-up.  All intermediate buffers live in one static
 * device array of 16 MiB inside the library (held by every GPU that loads
 * it, until exit); scenes, cameras and out_rgb are as for
 * pbr_render_forward.  Calls no cudaMalloc/cudaFree/cudaMallocAsync.
 *   - A pass that needs more than the 16 MiB (roughly: 56 B per point-view,
 *     8 B per pixel, 16 B per (tile, point-view) pair, plus sort scratch) is
 *     rejected with PBR_ERR_CAPACITY and a message giving the size needed;
 *     the check on pair counts happens after the per-point stage.
 *   - The first call on a device looks up the array's device address with
 *     cudaGetSymbolAddress (with that device current); make that first call
 *     before any stream capture.
 *   - Every call shares the array and it keeps the last call's contents
 *     (counters and tile ranges are cleared on each call); calls whose GPU
 *     work overlaps -- other streams or other host threads -- race on it.
 *   - Compositing is always one block per tile (opts->persistent is
 *     ignored: the persistent schedule's tile order would need more
 *     scratch); opts->batch_depth is honoured.
 *   - Synchronises the stream twice: once to size the lists, like
 *     pbr_render_forward, and once at the end to read the kernels' status
 *     word; a set status (e.g. more pairs than counted) returns
 *     PBR_ERR_DEVICE_STATUS. */
int pbr_render_forward_noalloc(const pbr_points *scenes, int32_t n_scenes,
                               const int32_t *scene_of_view, const pbr_camera *cams,
                               int32_t n_cams, const pbr_render_opts *opts, float *out_rgb,
                               pbr_stream_t stream);

/* ----------------------------------------- coarse-to-fine point update */
/* One pass of the hybrid coarse-to-fine update of Sec. 3.3 ("Hybrid
 * Coarse-to-Fine Updates") and Algorithm 1, which the paper runs between
 * training stages:
 *   1. voxel reduction: the cube anchored at the per-axis minimum of the
 *      positions, side = their largest per-axis extent, is split into
 *      n_vox^3 voxels; each non-empty voxel becomes one point whose
 *      parameters (position, SH, opacity, radius) are the means over the
 *      voxel's points.  Voxel of p: floor((p - lo) / h) per axis, h = side /
 *      n_vox, fp32 round-to-nearest, clamped; the reduced points come in
 *      ascending voxel id (z-major, x fastest).
 *   2. outlier removal: a reduced point is removed when the population
 *      standard deviation of the distances to its k nearest other reduced
 *      points exceeds eps (fp32, sums in neighbour order).  All points are
 *      judged against the same reduced set.
 *   3. point generation: every survivor adds one point whose parameters are
 *      the means over its k nearest other survivors.
 * Neighbours: ascending fp32 squared distance ((dx dx + dy dy) + dz dz),
 * ties by lower index; with fewer than k other points all of them are
 * used, and a point with none is kept (stage 2) and yields nothing
 * (stage 3).  Positions must be finite with magnitude below 1e18.
 *   in          : device arrays of the input cloud (pbr_points); the caller
 *                 keeps ownership; sh_degree fixes K = (sh_degree+1)^2.
 *   cfg->stages : bit 0 reduction, bit 1 outlier removal, bit 2 generation.
 *   out_*       : caller-owned device arrays with room for out_capacity
 *                 points ([cap,3], [cap,K,3], [cap], [cap]); they receive the
 *                 survivors in reduced order followed by the generated points
 *                 in the same order.  2 * in->n always suffices.
 *   counts      : host int64[3]: points after stage 1, after stage 2, and
 *                 in the output.
 * Errors: PBR_ERR_INVALID_ARG (null pointer, n_vox outside 1..1024, k
 * outside 1..32, eps negative or not finite, stages outside 0..7, n >=
 * 2^31); PBR_ERR_CAPACITY when the output needs more than out_capacity
 * points (counts are filled, nothing is written to out_*); PBR_ERR_OOM,
 * PBR_ERR_CUDA.  Synchronises the stream (the point counts are
 * data-dependent). */
typedef struct {
    int32_t n_vox;  /* voxels per axis (Algorithm 1 N), default 256 */
    int32_t k;      /* neighbours (Algorithm 1 K), default 8 */
    float eps;      /* threshold on the std of neighbour distances (Algorithm 1
                       epsilon), world units, default 0.01 */
    int32_t stages; /* default 7 (all three) */
} pbr_refine_cfg;
void pbr_default_refine(pbr_refine_cfg *cfg);
int pbr_refine_points(pbr_ctx *ctx, const pbr_points *in, const pbr_refine_cfg *cfg,
                      float *out_pos, float *out_sh, float *out_opacity, float *out_radius,
                      int64_t out_capacity, int64_t counts[3], pbr_stream_t stream);

/* Exact k nearest neighbours (the neighbour search of Algorithm 1, also
 * used for the point generation and frame initialisation of Sec. 3.3-3.4):
 * for each query point the k reference points of smallest fp32 squared
 * distance ((dx dx + dy dy) + dz dz), ties by lower index, ascending.
 *   ref_pos [n_ref,3], query_pos [n_query,3]: device, caller-owned.
 *   self     : 1 = the queries are the reference points (query_pos and
 *              n_query are ignored) and query i never returns point i.
 *   grid_n   : cells per axis of the search grid over the reference cube
 *              (1..1024), 0 = automatic (about 2 n_ref^(1/3)).
 *   out_idx [n_query,k] int32 and out_d2 [n_query,k] fp32 (device): rows
 *              padded with -1 / FLT_MAX past the available neighbours.
 * Errors: PBR_ERR_INVALID_ARG (k outside 1..32, grid_n outside 0..1024,
 * n_ref >= 2^31, null pointers), PBR_ERR_OOM, PBR_ERR_CUDA.  Asynchronous on
 * the stream. */
int pbr_knn(pbr_ctx *ctx, const float *ref_pos, int64_t n_ref, const float *query_pos,
            int64_t n_query, int32_t k, int32_t self, int32_t grid_n, int32_t *out_idx,
            float *out_d2, pbr_stream_t stream);

/* --------------------------------------------- video frame initialisation */
/* Chamfer distance between two clouds (the equation of Sec. 3.4, "Video
 * Synthesis"):
 *   CD = 1/n1 sum_i min_j |x_i - y_j|^2 + 1/n2 sum_j min_i |x_i - y_j|^2
 * and its gradient with respect to the second cloud's positions, with the
 * nearest points held fixed:
 *   dCD/dy_j = 2/n2 (y_j - x_nn(j)) + 2/n1 sum_{i: nn(i) = j} (y_j - x_i).
 * Nearest points by the exact neighbour search of pbr_knn (fp32 squared
 * distances, ties by lower index); distances in CD in fp64.
 *   p1 [n1,3], p2 [n2,3]: device, caller-owned, n1, n2 >= 1.
 *   loss_dev: device double, overwritten with CD.
 *   grad2 [n2,3] (device, nullable): overwritten with dCD/dp2.
 *   nn12 [n1], nn21 [n2] (device int32, nullable): the nearest-point maps.
 * Errors: PBR_ERR_INVALID_ARG, PBR_ERR_OOM, PBR_ERR_CUDA.  Asynchronous. */
int pbr_chamfer(pbr_ctx *ctx, const float *p1, int64_t n1, const float *p2, int64_t n2,
                double *loss_dev, float *grad2, int32_t *nn12, int32_t *nn21,
                pbr_stream_t stream);

/* Initialisation of a new frame from the trained previous one (Sec. 3.4):
 * `iters` Adam steps on the positions pos2 of the new cloud minimising the
 * Chamfer distance to the previous cloud, then every new point takes the
 * mean SH coefficients, opacity and radius of its k closest previous
 * points (the paper averages the SH "of the top-k closest points"; opacity
 * and radius are averaged the same way).  The paper gives no iteration
 * count, learning rate or k; the defaults are 100, 1e-3 and 4.
 *   prev   : the previous frame (device arrays, caller-owned, n >= 1).
 *   pos2   : [n2,3] device, updated in place (fp32 after every step).
 *   sh2 [n2,K,3] (K of prev->sh_degree), opacity2 [n2], radius2 [n2]:
 *            device, caller-owned, overwritten.
 *   loss_history: host double[iters + 1] (nullable): CD before every step
 *            and after the last one.
 * Errors: PBR_ERR_INVALID_ARG (null pointers, iters < 0, k outside 1..32,
 * lr negative or not finite, betas outside [0, 1), eps <= 0), PBR_ERR_OOM,
 * PBR_ERR_CUDA.  Synchronises the stream. */
typedef struct {
    int32_t iters;           /* Adam steps (default 100) */
    float lr;                /* learning rate (default 1e-3) */
    float beta1, beta2, eps; /* 0.9, 0.999, 1e-8 */
    int32_t k;               /* closest previous points per new point (default 4) */
    int32_t reserved[2];
} pbr_frame_cfg;
void pbr_default_frame_cfg(pbr_frame_cfg *cfg);
int pbr_frame_init(pbr_ctx *ctx, const pbr_points *prev, float *pos2, int64_t n2,
                   const pbr_frame_cfg *cfg, float *sh2, float *opacity2, float *radius2,
                   double *loss_history, pbr_stream_t stream);

/* ----------------------------------- visual hull and consistency check */
/* Consistency check of the paper's initialisation appendix (Sec. 3.1):
 * CC(p) = 1 iff p projects (Eq. 1) onto a foreground pixel of every view.
 * Projection in fp32 round-to-nearest, X = ((R0 px + R1 py) + R2 pz) + t
 * per row, u = fx (X.x / X.z) + cx, v = fy (X.y / X.z) + cy, pixel (floor
 * u, floor v); X.z <= z_near or a pixel outside the image is background.
 *   masks : device uint8, the views' [H, W] masks packed in camera order
 *           (> 0 = foreground), sum over views of W H bytes.
 *   keep  : device uint8 [n], overwritten with CC.
 * Errors: PBR_ERR_INVALID_ARG (null pointers, no camera, a camera of size
 * <= 0, z_near negative or not finite), PBR_ERR_OOM, PBR_ERR_CUDA.
 * Asynchronous. */
int pbr_consistency_check(pbr_ctx *ctx, const float *pos, int64_t n, const pbr_camera *cams,
                          int32_t n_cams, const uint8_t *masks, float z_near, uint8_t *keep,
                          pbr_stream_t stream);

/* The filter the paper applies after every training epoch: copies the
 * points with CC = 1, in order, to out_* (device, caller-owned, room for
 * in->n points) and writes their number to *n_out (host).  Errors as
 * pbr_consistency_check.  Synchronises the stream. */
int pbr_consistency_filter(pbr_ctx *ctx, const pbr_points *in, const pbr_camera *cams,
                           int32_t n_cams, const uint8_t *masks, float z_near, float *out_pos,
                           float *out_sh, float *out_opacity, float *out_radius, int64_t *n_out,
                           pbr_stream_t stream);

/* Visual-hull initialisation (Sec. 3.1): rejection sampling of uniform
 * points in the box [lo, hi) keeping those with CC = 1; the result is the
 * first n_target kept candidates of the counter-based stream `seed`.
 * Candidate j = lo + u (hi - lo) per axis (fp32, product then sum
 * rounded), u = the top 24 bits of SplitMix64 output 3 j + axis (Steele,
 * Lea and Flood 2014: output i of stream s is the generator's finaliser of
 * s + (i + 1) 0x9E3779B97F4A7C15) times 2^-24.  With out_sh set, the kept
 * points' SH coefficients ([n, (sh_degree+1)^2, 3], flattened index c) are
 * standard normals by Box-Muller (fp32 logf and sincospif: no decision
 * depends on them) on stream seed ^ 0x5DEECE66D,
 * pair c / 2 from outputs c - c % 2 and c - c % 2 + 1 (even c: cosine,
 * odd: sine; u1 = (top 24 bits + 1) 2^-24).
 *   out_pos [n_target,3] (device, caller-owned); out_sh nullable.
 *   max_candidates: candidates drawn at most (0 = 2^40).
 *   *n_out: points kept (< n_target when the limit was reached first);
 *   *n_drawn: candidates drawn up to and including the last kept one.
 * Errors: PBR_ERR_INVALID_ARG (as above, a box with hi < lo or not finite,
 * n_target outside 0..2^31-1, sh_degree outside 0..3), PBR_ERR_OOM,
 * PBR_ERR_CUDA.  Synchronises the stream. */
int pbr_visual_hull_init(pbr_ctx *ctx, const float lo[3], const float hi[3],
                         const pbr_camera *cams, int32_t n_cams, const uint8_t *masks,
                         float z_near, uint64_t seed, int64_t n_target, int64_t max_candidates,
                         int32_t sh_degree, float *out_pos, float *out_sh, int64_t *n_out,
                         int64_t *n_drawn, pbr_stream_t stream);

/* ------------------------------------------------------- microbenchmarks */
/* Measures the device's FP32 FMA rate (flop/s, an FMA counted as 2) and
 * MUFU ex2 rate (op/s) with the library's own kernels; used as the ALU
 * roofline of the raster kernels.  Synchronises. */
int pbr_measure_alu_peaks(int device, double *fp32_flops, double *ex2_ops);

#ifdef __cplusplus
}
#endif
#endif /* PBR_H */
