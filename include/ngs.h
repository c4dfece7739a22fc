/*
 * ngs.h -- C ABI of the GB300 (sm_103a) library for generalized non-exponential Gaussian splatting.
 *
 * The library renders a set of 3D Gaussians through a pinhole camera by front-to-back compositing of
 * depth-sorted splats under a mother transmittance T(tau) (Sec. 4.2, Eq. generalized_gaussian and
 * Eq. nexp_p; the per-model slope terms of Table 1), stopping each ray once its transmittance
 * saturates, and differentiates the result by path replay (Sec. 5.1 "Optimization"; App. C).
 *
 * Conventions shared by every call:
 *  - All array arguments are DEVICE pointers owned by the caller (for example PyTorch tensors), FP32
 *    unless stated, densely packed, row-major. The library never frees them.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default stream. Every kernel of a
 *    call is launched on that stream; a call returns before its kernels finish, except where a call
 *    documents one host synchronisation.
 *  - Return value: NGS_OK (0) or a negative NGS_ERR_* status. On error nothing is launched that would
 *    write caller memory after the return, and ngs_last_error() holds a one-line message. No C++
 *    exception crosses this boundary.
 *  - A context (ngs_ctx) is not thread-safe: use one per host thread / stream. A frame (ngs_frame)
 *    belongs to the context that created it.
 */
#ifndef NGS_H
#define NGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define NGS_API __attribute__((visibility("default")))
#else
#define NGS_API
#endif

/* ---- status codes ---------------------------------------------------------------------------- */
#define NGS_OK 0
#define NGS_ERR_INVALID_ARG (-1)   /* a pointer, size or option is out of its documented range      */
#define NGS_ERR_OUT_OF_MEMORY (-2) /* device allocation of internal buffers failed                  */
#define NGS_ERR_CUDA (-3)          /* a CUDA runtime call failed (message in ngs_last_error)       */
#define NGS_ERR_DEVICE_CHECK (-5)  /* a kernel's own bounds check fired (in this or an earlier call   */
                                   /* on the context; reported at the next render); that output was  */
                                   /* not valid                                                       */
#define NGS_ERR_CAPACITY (-6)      /* an asynchronous render met more (tile, Gaussian) pairs than its */
                                   /* frame's capacity: its output is not valid; the capacity has     */
                                   /* grown, so rendering again succeeds (ngs_frame_status)           */

/* ---- transmittance models (Table 1) ----------------------------------------------------------- */
#define NGS_MODEL_EXP 0  /* T = exp(-tau): pbar_i = alpha_i prod_{j<i}(1 - alpha_j) (standard 3DGS)      */
#define NGS_MODEL_QUAD 1 /* T = [1 - tau - c/2 tau^2]_+: pbar_i = alpha_i (1 + c taubar_i); param = c,    */
                         /* c >= -1/2. c = -1/2 sub-linear, c = 0 linear, c = +1/2 super-linear (Sec. 5)  */
#define NGS_MODEL_BLEND 2  /* T = [lerp(1 - tau, exp(-tau), g)]_+: pbar_i = alpha_i (1 - g + g P_i),        */
                           /* P_i = prod_{j<i}(1 - alpha_j); param = g in [0, 1]                          */
#define NGS_MODEL_VICINI 3 /* T = lerp([1 - tau]_+, exp(-tau), g): pbar_i = lerp(pbar_i^lin, pbar_i^exp, g), */
                           /* each list with its own stop (linear: saturation; exponential: t_eps);       */
                           /* the ray stops when both have; param = g in [0, 1]                           */

typedef struct ngs_ctx ngs_ctx;
typedef struct ngs_frame ngs_frame;

/* Gaussian parameters (Sec. 3: centre c_i, covariance Sigma_i, opacity aleph_i, emission E_i(omega)).
 * Raw parametrisation: Sigma_i = R(q) diag(exp(2 s)) R(q)^T with q = quats[i] normalised inside the
 * library (w, x, y, z order), aleph_i = sigmoid(opacity_logits[i]),
 * E_i = max(0, 1/2 + sum_lm Y_lm(d) sh[i][lm]) per colour channel, Y_lm the real spherical harmonics of
 * degree <= sh_degree in the coefficient order of 3D Gaussian splatting assets, d the unit direction
 * from the camera centre to the mean. */
typedef struct {
  int64_t n;                   /* number of Gaussians, 0 <= n < 2^31                                  */
  int32_t sh_degree;           /* 0..3                                                              */
  const float* means;          /* [n][3] world position                                             */
  const float* log_scales;     /* [n][3] s                                                          */
  const float* quats;          /* [n][4] (w, x, y, z), nonzero norm                                 */
  const float* opacity_logits; /* [n]                                                               */
  const float* sh;             /* [n][(sh_degree + 1)^2][3]                                         */
} ngs_gaussians;

/* Pinhole camera looking down +z of its view frame. Pixel (x, y) samples the image point
 * (x + 1/2, y + 1/2); a view-space point (X, Y, Z) maps to (fx X / Z + cx, fy Y / Z + cy). */
typedef struct {
  float viewmat[12]; /* world -> view, row-major [R | t] (3 x 4); R must be a rotation                */
  float fx, fy, cx, cy;
  int32_t width, height; /* 1 .. 16384                                                              */
} ngs_camera;

typedef struct {
  int32_t kind; /* NGS_MODEL_EXP, _QUAD, _BLEND or _VICINI (Table 1)                                   */
  float param;  /* c for NGS_MODEL_QUAD (>= -0.5), g for _BLEND / _VICINI (0..1); ignored for _EXP      */
} ngs_model;

/* Rendering options. ngs_default_options() fills the values below, which are the conventions of the
 * 3D Gaussian splatting baseline the paper builds on (the paper itself states none of them). */
typedef struct {
  float alpha_min;     /* 1/255: a splat with alpha_i(p) < alpha_min is skipped at pixel p           */
  float alpha_max;     /* 0.99: alpha_i(p) = min(alpha_max, aleph_i K_i(p))                          */
  float t_eps;         /* 1e-4: exponential model only, stop before T would fall below t_eps         */
  float dilation;      /* 0.3: added to the 2D covariance's diagonal, in pixel^2                     */
  float near_plane;    /* 0.2: Gaussians with FP32 view depth <= near_plane are culled               */
  float background[3]; /* L_b of Eq. generalized_gaussian; default black                             */
  int32_t tile_w, tile_h; /* screen tile: 8x8, 16x16 (default) or 16x32; the image does not depend on it */
  int32_t max_splats;  /* 0 = unlimited, else at most this many splats composited per pixel (the    */
                       /* paper's ray tracer caps at 128, Sec. 5.1 "Renderer")                       */
  int32_t chunk;       /* splat records staged in shared memory per round of a tile's list walk:      */
                       /* 0 = the tile's pixel count (default), else half, equal to or twice it       */
  int32_t schedule;    /* NGS_SCHEDULE_TILES (default) or NGS_SCHEDULE_PERSISTENT                     */
} ngs_options;         /* tile shape, chunk and schedule change the speed, never the results          */

/* Composite schedules: one CTA per screen tile in tile order, or one wave of persistent CTAs that take
 * tiles from a list ordered by descending (tile, splat) pair count, so that the longest tiles start first. */
#define NGS_SCHEDULE_TILES 0
#define NGS_SCHEDULE_PERSISTENT 1

/* Gradient outputs of ngs_render_backward, same shapes as ngs_gaussians' arrays. OVERWRITTEN. */
typedef struct {
  float* d_means;
  float* d_log_scales;
  float* d_quats;
  float* d_opacity_logits;
  float* d_sh;
} ngs_grads;

/* Read-only view of a frame's buffers (valid until the frame's next render or destruction). A frame
 * rendered from n_views cameras (ngs_render_batch) packs its views one after the other: splat record
 * r = v n + i belongs to view v and Gaussian i; view v's tiles have the global indices
 * [view_tile_base[v], view_tile_base[v + 1]) (local tile ty * tiles_x_v + tx), and its pixels the packed
 * indices [view_pixel_base[v], view_pixel_base[v + 1]) (local pixel y * width_v + x). */
typedef struct {
  int64_t n_gaussians;
  int64_t n_pairs;          /* number of (tile, splat record) pairs after binning                     */
  int32_t tiles_x, tiles_y; /* of view 0                                                              */
  int32_t width, height;    /* of view 0                                                              */
  float log2_alpha_min;     /* FP32 threshold of the alpha test on the exponent                       */
  int32_t n_views;
  const float* records;     /* device [n_views n][12] splat records: u, v, A', B', C', L, E0, E1, E2,  */
                            /*   z, rx, ry with (A', B', C') = -log2(e)/2 (A, 2B, C) of the conic,      */
                            /*   L = log2 aleph, z the FP32 view depth, (rx, ry) the half extents of   */
                            /*   the alpha >= alpha_min ellipse's bounding box (0: no tile)            */
  const uint64_t* keys;     /* device [n_pairs] sorted keys (global tile << 32) | bits(z)             */
  const uint32_t* values;   /* device [n_pairs] splat record index of each key                        */
  const uint32_t* ranges;   /* device [tiles][2] [start, end) of each global tile's pairs             */
  const float* pixel_state; /* device [pixels][8] replay state written by the forward pass            */
  const int64_t* view_pixel_base; /* HOST [n_views + 1]                                               */
  const uint32_t* view_tile_base; /* HOST [n_views + 1]                                               */
} ngs_frame_view;

/* Fill `out` with the default options above. */
NGS_API void ngs_default_options(ngs_options* out);

/* Create a context on the current CUDA device. *out receives the handle. Returns NGS_ERR_CUDA if no
 * device is usable. */
NGS_API int ngs_create(ngs_ctx** out);

/* Destroy a context (frees its scratch memory after synchronising the device). NULL is allowed. */
NGS_API void ngs_destroy(ngs_ctx* ctx);

/* One-line description of the last error on this context ("" if none). Owned by the context. */
NGS_API const char* ngs_last_error(const ngs_ctx* ctx);

/* A frame holds everything one render leaves for its backward pass: splat records, sorted
 * (tile, Gaussian) pairs, tile ranges and the per-pixel replay state (the paper's path replay passes
 * E_k from the forward to the adjoint pass, App. C.1). Its buffers are allocated and grown by the
 * library on first use and reused by later renders into the same frame. */
NGS_API int ngs_frame_create(ngs_ctx* ctx, ngs_frame** out);
NGS_API void ngs_frame_destroy(ngs_frame* frame);

/* Asynchronous renders into a frame (off by default). With `enable` set, ngs_render and ngs_render_batch
 * into this frame enqueue the whole pipeline without the host synchronisation after binning: the pair
 * buffers are sized from the frame's pair capacity (the largest pair count its earlier renders met, plus a
 * quarter) and the kernels after binning read the count from device memory. A render whose count exceeds
 * the capacity writes only the pairs that fit, so its image and replay state are not valid; it is reported
 * by ngs_frame_status. A frame without a capacity yet (no earlier render) renders synchronously, which sets
 * one. Results of a render that fits are bit-identical to the synchronous render.
 * Errors: NGS_ERR_INVALID_ARG for a NULL frame. */
NGS_API int ngs_frame_set_async(ngs_frame* frame, int enable);

/* Waits for the frame's last render and reports every render into the frame since the previous call:
 * NGS_OK; NGS_ERR_CAPACITY if an asynchronous one exceeded the frame's pair capacity (the capacity then
 * grows to the count met plus a quarter, so rendering again succeeds); NGS_ERR_DEVICE_CHECK if a kernel
 * bounds check fired. *pairs (may be NULL) receives the last render's pair count. Clears what it reports.
 * Errors: NGS_ERR_INVALID_ARG for a NULL frame or a frame that holds no render; NGS_ERR_CUDA. */
NGS_API int ngs_frame_status(ngs_frame* frame, int64_t* pairs);

/* Render (Eq. generalized_gaussian with pbar_i from Eq. nexp_p):
 *   image[y][x][3] = sum_i E_i pbar_i + L_b Tbar_end over the splats i of pixel (x, y), front to back by
 *   (FP32 view depth, Gaussian index); overdraw[y][x] = number of splats composited at that pixel,
 *   the saturating one included (Fig. 2 "Overdraws"; Table 3 "Avg. OD").
 * `image` is [height][width][3] FP32 and `overdraw` [height][width] int32, both caller-owned device
 * memory; overdraw may be NULL. The frame is overwritten. One host synchronisation happens after
 * binning, to read the number of (tile, Gaussian) pairs and size the sort buffers (none for a frame in
 * asynchronous mode that has a capacity, see ngs_frame_set_async).
 * Errors: NGS_ERR_INVALID_ARG for NULL pointers, n < 0, sh_degree outside 0..3, width/height outside
 * 1..16384, an unsupported tile shape, chunk or schedule, kind/param outside the table above. */
NGS_API int ngs_render(ngs_ctx* ctx, ngs_frame* frame, const ngs_gaussians* g, const ngs_camera* cam,
                       const ngs_model* model, const ngs_options* opt, float* image, int32_t* overdraw,
                       void* stream);

/* Render one set of Gaussians from n_views cameras (1 <= n_views <= 4096) of any sizes in one pass of the
 * pipeline: one projection launch for all (view, Gaussian) pairs, in which the views of a block of
 * Gaussians run side by side so the parameters are read from HBM once; one segmented depth sort; one
 * binning into global tiles (view v's tiles follow those of views 0..v-1); one tile sort; one composite
 * launch over the tiles of all views. Each view's image and overdraw are bit-identical to ngs_render of
 * that camera alone with the same options (the same per-tile splat lists and arithmetic).
 * `cams` is a HOST array [n_views]. `images` packs the views one after the other: view v occupies pixels
 * [P_v, P_v + H_v W_v) with P_v = sum_{u<v} H_u W_u, so images is [sum H_v W_v][3] and overdraw (may be
 * NULL) [sum H_v W_v]. One host synchronisation, as in ngs_render. n * n_views must be below 2^32.
 * ngs_render_backward of a batch frame takes dl_dimage packed the same way and writes the gradient of the
 * sum over the views. Errors: those of ngs_render, and n_views out of range. */
NGS_API int ngs_render_batch(ngs_ctx* ctx, ngs_frame* frame, const ngs_gaussians* g, const ngs_camera* cams,
                             int32_t n_views, const ngs_model* model, const ngs_options* opt, float* images,
                             int32_t* overdraw, void* stream);

/* Path-replay backward of the frame's last render (App. C: recursive adjoints computed front to back by
 * replaying each pixel's splat list, recomputing alpha_i and taubar_i instead of storing per-splat state).
 * dl_dimage: [height][width][3] FP32 device array (dL/dL0 per pixel). `g` must hold the same parameter
 * values the frame was rendered from. Gradients w.r.t. the raw parameters are written (not accumulated)
 * into `out`; Gaussians that were culled get zeros. Errors: NGS_ERR_INVALID_ARG if the frame holds no
 * render or `g` does not match its size. */
NGS_API int ngs_render_backward(ngs_ctx* ctx, const ngs_frame* frame, const ngs_gaussians* g,
                                const float* dl_dimage, const ngs_grads* out, void* stream);

/* The backward above, for callers that cannot let the library allocate device memory (an application
 * that owns a fixed device-memory budget, or a latency-critical loop where cudaMalloc / cudaFree would
 * synchronise the device). The paper has no counterpart: this is an interface addition. Same arguments
 * and results as ngs_render_backward, but the per-Gaussian scratch lives in one static device array of
 * 12 MiB that every GPU loading the library holds until the process exits, and nothing is allocated.
 * Limits: at most 262,144 splat records, Gaussians x views (larger frames return NGS_ERR_INVALID_ARG with
 * a message naming the limit). All calls on a device share the array; each call clears what it uses first, and calls that
 * overlap on the GPU (unordered streams or threads) race on it. The context's device must be the current
 * device (else NGS_ERR_INVALID_ARG). The first call on a device looks up the array's address there
 * (cudaGetSymbolAddress); make it before any stream capture. */
NGS_API int ngs_render_backward_static(ngs_ctx* ctx, const ngs_frame* frame, const ngs_gaussians* g,
                                       const float* dl_dimage, const ngs_grads* out, void* stream);

/* Fill `out` with pointers into the frame (for tests and diagnostics). The render path sorts 32-bit tile
 * indices only (the splats are already in depth order); this call composes the 64-bit keys from them and
 * the records, and synchronises the device to do so. */
NGS_API int ngs_frame_view_get(const ngs_frame* frame, ngs_frame_view* out);

/* CUDA graphs (off by default). When enabled, ngs_render and ngs_render_batch run each of their two phases
 * (projection .. pair count; key emission .. composite) as a CUDA graph, captured on the context's own
 * stream the first time a frame meets a configuration (Gaussian arrays, image sizes, model, options,
 * output pointers) and replayed after that. Camera poses are copied in by the graph, so a new pose needs
 * no new capture; phase 2 is captured for a pair capacity (the count met plus a quarter) that replays reuse
 * while the count fits, its kernels reading the exact count from device memory. Results are bit-identical
 * to the direct launches. Stage timing is not recorded for replayed phases. ngs_graph_captures returns how
 * many phases the context has captured. */
NGS_API int ngs_set_graphs(ngs_ctx* ctx, int enable);
NGS_API int64_t ngs_graph_captures(const ngs_ctx* ctx);

/* Autotuner. Times the render (and, when dl_dimage and grads are both given, the backward too) of this
 * batch under every supported launch configuration -- tile shape 8x8, 16x16, 16x32; chunk half, once and
 * twice the tile's pixel count; schedule tiles or persistent -- and writes the fastest into *best, every
 * other field copied from *base. Each candidate gets one untimed render (+ backward) and then `reps`
 * (1..100) timed ones, CUDA events on `stream` around each; a candidate's time is the median. When
 * flush_bytes > 0, a context-owned scratch of that size is cleared before each timed call (outside the
 * events), so that no candidate finds its inputs in L2 left over from the previous call. The results
 * of a render never depend on these choices, only its speed. `table` (may be NULL) receives one entry per
 * candidate, up to table_cap. Returns the number of candidates timed, or a negative status.
 * Synchronises the stream; the frame holds the last candidate's render afterwards. Arguments otherwise as
 * ngs_render_batch and ngs_render_backward. */
typedef struct {
  int32_t tile_w, tile_h, chunk, schedule;
  float ms; /* median time of one render (+ backward), milliseconds */
} ngs_tune_entry;
NGS_API int ngs_autotune(ngs_ctx* ctx, ngs_frame* frame, const ngs_gaussians* g, const ngs_camera* cams,
                         int32_t n_views, const ngs_model* model, const ngs_options* base, float* images,
                         int32_t* overdraw, const float* dl_dimage, const ngs_grads* grads, int32_t reps,
                         int64_t flush_bytes, ngs_options* best, ngs_tune_entry* table, int32_t table_cap,
                         void* stream);

/* Stage timing. When enabled, every render/backward records CUDA events on its stream around each
 * stage and ngs_stage_times() adds up the elapsed time per stage (synchronising on the recorded
 * events). Stages: 0 project, 1 depth sort, 2 scan + key emit, 3 tile sort, 4 tile ranges,
 * 5 composite forward, 6 composite backward (replay), 7 projection backward. `ms` and `launches` have
 * room for `n` entries; returns the number of stages. ngs_reset_stage_times() clears the sums. */
#define NGS_NUM_STAGES 8
NGS_API int ngs_set_timing(ngs_ctx* ctx, int enable);
NGS_API int ngs_stage_times(ngs_ctx* ctx, double* ms, int64_t* launches, int32_t n);
NGS_API void ngs_reset_stage_times(ngs_ctx* ctx);

/* Total number of kernel launches this context has issued (all stages). */
NGS_API int64_t ngs_launch_count(const ngs_ctx* ctx);

/* ---- memory planning and checked mode ------------------------------------------------------------- */

/* Device memory that a render of n Gaussians from n_views cameras (and its backward) allocates in a fresh
 * context and frame, for admission control before the render. A frame keeps its buffers and grows them
 * by at least a quarter when a later render needs more; a context likewise.
 *   frame_fixed     the frame's buffers sized by splat records, tiles and pixels: records (48 B per record),
 *                   tile counts, depth keys and order (ping-pong), scan offsets, tile ranges, the per-pixel
 *                   replay state (32 B per pixel), the view table, and the persistent schedule's work list;
 *   frame_pairs     the frame's pair buffers (tile and record index, ping-pong: 16 B per pair) for n_pairs;
 *   context         the context's scratch for this render: radix histograms of both sorts, scan block sums
 *                   and the pair-count word;
 *   backward        the context's per-record gradient scratch of ngs_render_backward (48 B per record);
 *   total           their sum.
 * n_pairs is the number of (tile, splat) pairs the pair buffers are sized for: the exact count for a
 * synchronous render without graphs, else the frame's capacity (count + count / 4 + 1024). Every size is
 * rounded up as the library's allocations are (to 256 B). Errors: NGS_ERR_INVALID_ARG as ngs_render_batch
 * for the cameras and options, n < 0 or n_pairs < 0. No device call is made. */
typedef struct {
  size_t frame_fixed, frame_pairs, context, backward, total;
} ngs_workspace;
NGS_API int ngs_workspace_bytes(int64_t n, const ngs_camera* cams, int32_t n_views, const ngs_options* opt,
                                int64_t n_pairs, ngs_workspace* out);

/* Device bytes a context and a frame hold now (either may be NULL; its count is then 0). */
NGS_API int ngs_memory_usage(const ngs_ctx* ctx, const ngs_frame* frame, size_t* ctx_bytes, size_t* frame_bytes);

/* Checked mode (off by default): every render on the context first scans the Gaussian parameters and,
 * when any is NaN or infinite, returns NGS_ERR_INVALID_ARG naming the array, having launched nothing
 * else. The fast path does not scan; the scan reads each parameter once and synchronises the host with
 * the stream (an asynchronous frame's render is then no longer free of host synchronisation). */
NGS_API int ngs_set_checked(ngs_ctx* ctx, int enable);

/* ---- roofline denominators --------------------------------------------------------------------------
 * Throughput of the pipes the compositing kernels are bound by, measured on the context's device: eight
 * independent dependency chains per thread on every SM at full occupancy, timed with CUDA events on
 * `stream` over about `seconds` (0.01 .. 60) of work; *rate receives the best of four timed launches.
 * Synchronises the stream. The paper has no counterpart: this is a measurement aid. */
#define NGS_PEAK_FFMA 0  /* fma.rn.f32: FLOP/s, an FMA counting 2                                        */
#define NGS_PEAK_FFMA2 1 /* fma.rn.f32x2 (two lanes per instruction): FLOP/s, an FMA counting 2 per lane  */
#define NGS_PEAK_EX2 2   /* ex2.approx.ftz.f32 (MUFU): results per second                                 */
NGS_API int ngs_measure_peak(ngs_ctx* ctx, int32_t kind, double seconds, double* rate, void* stream);

/* ---- training step (Sec. 5.1 "Loss", "Optimization", "Densification") -------------------------------- */

/* Image loss L = (1 - lambda) L1 + lambda (1 - SSIM) of `image` against `target` (both device
 * [height][width][3] FP32): L1 the mean absolute difference, SSIM the mean over pixels and channels of the
 * structural similarity of Wang et al. with the 11 x 11 Gaussian window (sigma 1.5), C1 = 0.01^2,
 * C2 = 0.03^2 and zero padding, as in 3D Gaussian splatting. dl_dimage (device, may be NULL) receives
 * dL/dimage. loss_out (host double[3], may be NULL) receives (L, L1, SSIM); it synchronises the stream. */
NGS_API int ngs_loss_l1_ssim(ngs_ctx* ctx, const float* image, const float* target, int32_t width, int32_t height,
                             float lambda, float* dl_dimage, double* loss_out, void* stream);

/* Adam over the five parameter arrays of n Gaussians (ngs_grads layout: means, log_scales, quats,
 * opacity_logits, sh) in one launch, with per-array learning rates lr[5]: m = b1 m + (1 - b1) g,
 * v = b2 v + (1 - b2) g^2, theta -= lr m^ / (sqrt(v^) + eps) with the bias corrections of step `step`
 * (1-based). bounded != 0 clips each update to [-lr, lr] (the paper's "bounded Adam" as read here). */
typedef struct {
  float lr[5];
  float beta1, beta2, eps;
  int32_t step;
  int32_t bounded;
} ngs_adam;
NGS_API int ngs_adam_step(ngs_ctx* ctx, int64_t n, int32_t sh_degree, const ngs_grads* params,
                          const ngs_grads* grads, const ngs_grads* m, const ngs_grads* v, const ngs_adam* cfg,
                          void* stream);

/* accum[i] += |d_means[i]| and count[i] += 1 for every Gaussian with a nonzero positional gradient. */
NGS_API int ngs_accumulate_grad_norm(ngs_ctx* ctx, int64_t n, const float* d_means, float* accum, float* count,
                                     void* stream);

/* Split / prune (Sec. 5.1 "Densification"). Gaussian i is pruned (prune != 0) when its opacity is below
 * min_opacity or its largest scale below min_scale; else split (split != 0) when accum[i] / count[i] >
 * grad_threshold; else kept. Splits are granted in index order while the count stays within max_gaussians.
 * A split writes two children at mu +- (sigma_a / 2) r_a along the longest axis a, with sigma_a scaled by
 * sqrt(3)/2 (the pair keeps the parent's variance along r_a) and everything else the parent's; kept
 * Gaussians keep their Adam moments, children start from zero. Writes the surviving and new Gaussians, in
 * index order, to out_* (capacity >= min(2 n, max(n, max_gaussians))) and their number to *n_out
 * (host); synchronises the stream. n < 2^30. */
typedef struct {
  float grad_threshold;
  float min_opacity;
  float min_scale;
  int32_t split;
  int32_t prune;
  int64_t max_gaussians;
} ngs_densify_cfg;
NGS_API int ngs_densify(ngs_ctx* ctx, int64_t n, int32_t sh_degree, const ngs_grads* params, const ngs_grads* m,
                        const ngs_grads* v, const float* accum, const float* count, const ngs_densify_cfg* cfg,
                        int64_t capacity, const ngs_grads* out_params, const ngs_grads* out_m,
                        const ngs_grads* out_v, int64_t* n_out, void* stream);

/* ---- render server ---------------------------------------------------------------------------------
 * A request loop over scenes kept resident on the device. The paper has no counterpart: this is the
 * serving form of the render call above.
 *  - Workers: `workers` host threads, each with its own CUDA stream, context and frame, so batches of
 *    different workers overlap on the device.
 *  - Continuous batching: a free worker takes the oldest pending request together with every pending
 *    request for the same scene and model (in arrival order, at most max_batch_views) and renders them as
 *    one ngs_render_batch-style pass; requests that arrive while the GPU is busy join the next batch.
 *    Each image equals ngs_render of that request alone, bit for bit.
 *  - Admission by memory: a batch reserves the bytes ngs_workspace_bytes reports for it -- frame_fixed +
 *    context before it starts, frame_pairs once the exact pair count is known; it waits while the
 *    reservations of the batches in flight would exceed mem_budget. The oldest batch in flight may always
 *    proceed (counted in over_budget_admissions when that exceeds the budget), so one always progresses.
 * Threading: submit, poll and get_stats may be called from any host thread. Requests reference caller-owned
 * device memory (scene arrays, output images) that must stay valid until the request completes. */
typedef struct ngs_server ngs_server;

typedef struct {
  int32_t workers;         /* 1..64 (default 4)                                                        */
  int32_t max_batch_views; /* 1..4096 (default 16)                                                     */
  int64_t mem_budget;      /* bytes all batches in flight may reserve (default 8 GiB)                  */
  int32_t graphs;          /* 1: workers capture/replay CUDA graphs of the render phases; 0 (default):  */
                           /* direct launches (batch shapes vary, so replays rarely match a capture)   */
  int32_t reserved;        /* 0                                                                         */
  ngs_options options;     /* render options of every request (default: ngs_default_options)           */
} ngs_server_config;

typedef struct {
  int32_t scene;        /* id returned by ngs_server_add_scene                                          */
  ngs_model model;
  ngs_camera camera;
  float* image;         /* device [height][width][3], written when the request completes                */
  int32_t* overdraw;    /* device [height][width] or NULL                                               */
  int64_t tag;          /* the caller's identifier, returned in the completion                          */
} ngs_request;

typedef struct {
  int64_t tag;
  int32_t status;       /* NGS_OK or the error of its batch                                             */
  int32_t batch_views;  /* number of requests in its batch                                              */
  double submit_s;      /* server clock (seconds since creation): submission, batch start, completion   */
  double start_s;       /* (images on the device and the stream synchronised)                           */
  double done_s;
  int64_t pairs;        /* (tile, splat) pairs of its batch                                             */
} ngs_completion;

typedef struct {
  int64_t submitted, completed, batches, max_batch_views;
  int64_t over_budget_admissions;
  int64_t peak_reserved_bytes, reserved_bytes, pending;
  double now_s;
} ngs_server_stats;

NGS_API void ngs_default_server_config(ngs_server_config* cfg);
/* Starts the workers on the current device. Errors: NGS_ERR_INVALID_ARG for values out of range. */
NGS_API int ngs_server_create(const ngs_server_config* cfg, ngs_server** out);
/* Register a resident scene (the arrays are referenced, not copied); *id receives its id. */
NGS_API int ngs_server_add_scene(ngs_server* server, const ngs_gaussians* g, int32_t* id);
/* Queue a request; returns at once. A camera or model outside its documented range is refused here with
 * NGS_ERR_INVALID_ARG (it never joins a batch); errors met while rendering are reported in the
 * completions of the batch's requests. */
NGS_API int ngs_server_submit(ngs_server* server, const ngs_request* request);
/* Move up to `cap` completions to `out`, waiting up to wait_ms for the first; returns how many. */
NGS_API int ngs_server_poll(ngs_server* server, ngs_completion* out, int32_t cap, int32_t wait_ms);
NGS_API int ngs_server_get_stats(ngs_server* server, ngs_server_stats* out);
/* The first error a batch met ("" if none). */
NGS_API const char* ngs_server_last_error(ngs_server* server);
/* Render every queued request, then stop the workers and free the server. */
NGS_API void ngs_server_destroy(ngs_server* server);

#ifdef __cplusplus
}
#endif

#endif /* NGS_H */
