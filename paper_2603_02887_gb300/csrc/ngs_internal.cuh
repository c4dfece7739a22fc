// Internal declarations shared by the CUDA translation units of the ngs library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ngs.h"

namespace ngs {

// ---- launch-time constants passed by value to kernels ------------------------------------------

struct CamParams {
  float R[9];       // world -> view rotation, row-major
  float t[3];
  float fx, fy, cx, cy;
  float campos[3];  // camera centre in world space, -R^T t
  int W, H;
};

// One view of a batch (a device array of these per frame). Views are packed one after the other: view v's
// splat records are records [v n, (v + 1) n), its tiles have the global indices [tile_base, tile_base +
// tiles_x tiles_y) and its pixels the packed indices [pix_base, pix_base + W H) of the replay state. Its
// image and overdraw map are written to `image` / `overdraw` (row-major [H][W][3] / [H][W]).
struct ViewParams {
  CamParams cam;
  int tiles_x, tiles_y;
  uint32_t tile_base;
  uint32_t pad;
  uint64_t pix_base;
  float* image;
  int32_t* overdraw;  // may be null
};

struct RenderParams {
  float alpha_min, alpha_max, t_eps, dilation, near_plane;
  float log2_alpha_min;  // the alpha >= alpha_min test is made on log2(alpha)
  float bg[3];
  float c;               // model parameter: c (quadratic) or gamma (blended, Vicini)
  float c1;              // 1 - gamma
  int kind;
  int tile_w, tile_h;
  int tiles_x, tiles_y;  // of the view a kernel works on (kernels that see several views set them per view)
  int width, height;     // of view 0
  int max_splats;
  int chunk;             // records staged per round of a tile's list walk (tile pixels x 1/2, 1 or 2)
  int schedule;          // NGS_SCHEDULE_*
  int cam_from_table;    // the projection reads every camera from the view table (else a single view's
                         // camera is a kernel parameter)
  int sh_degree;
  uint32_t n_gaussians;  // n: Gaussians per view
  uint32_t n_views;
  uint32_t n_records;    // n_views * n: splat records (and valid pair values)
  uint32_t n_tiles;      // tiles of all views
  uint32_t* check;       // device error word: kernels OR in a kCheck* bit when a bounds check fires
};

constexpr uint32_t kCheckIndex = 1u;     // a sorted pair named a splat record index >= n_records
constexpr uint32_t kCheckCapacity = 2u;  // an asynchronous render met more pairs than its capacity
constexpr uint32_t kCheckTile = 8u;      // a sorted pair named a tile outside the batch's tiles

// Geometry of the view holding global tile t. A single view takes it from the kernel parameters (no
// dependent load before the tile's work starts); a batch looks it up in the view table.
struct TileView {
  int view;                  // index of the view (0 for a single view)
  int W, H, tiles_x, local;  // image size, tiles per row, tile index within the view
};

__device__ __forceinline__ int view_of_tile(const ViewParams* __restrict__ views, int n_views, uint32_t t);

__device__ __forceinline__ TileView tile_view(const RenderParams& rp, const ViewParams* __restrict__ views,
                                              uint32_t t) {
  TileView tv;
  if (rp.n_views == 1) {
    tv.view = 0;
    tv.W = rp.width;
    tv.H = rp.height;
    tv.tiles_x = rp.tiles_x;
    tv.local = (int)t;
  } else {
    const int v = view_of_tile(views, (int)rp.n_views, t);
    tv.view = v;
    tv.W = __ldg(&views[v].cam.W);
    tv.H = __ldg(&views[v].cam.H);
    tv.tiles_x = __ldg(&views[v].tiles_x);
    tv.local = (int)(t - __ldg(&views[v].tile_base));
  }
  return tv;
}

// First packed pixel (replay state) and output arrays of view v; a single view takes its outputs from the
// kernel parameters. Looked up where they are used, so that they are not held in registers meanwhile.
__device__ __forceinline__ size_t view_pix_base(const RenderParams& rp, const ViewParams* __restrict__ views, int v) {
  return rp.n_views == 1 ? 0 : (size_t)__ldg(reinterpret_cast<const unsigned long long*>(&views[v].pix_base));
}
__device__ __forceinline__ float* view_image(const RenderParams& rp, const ViewParams* __restrict__ views, int v,
                                             float* image0) {
  return rp.n_views == 1 ? image0
                         : reinterpret_cast<float*>(__ldg(reinterpret_cast<const unsigned long long*>(&views[v].image)));
}
__device__ __forceinline__ int32_t* view_overdraw(const RenderParams& rp, const ViewParams* __restrict__ views, int v,
                                                  int32_t* overdraw0) {
  return rp.n_views == 1
             ? overdraw0
             : reinterpret_cast<int32_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&views[v].overdraw)));
}

// The view whose global tiles contain tile t (views[0].tile_base = 0; tile bases ascend).
__device__ __forceinline__ int view_of_tile(const ViewParams* __restrict__ views, int n_views, uint32_t t) {
  int lo = 0, hi = n_views - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(&views[mid].tile_base) <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Splat record: 3 float4 per Gaussian.
//   r0 = (u, v, A', B'), r1 = (C', L, E0, E1), r2 = (E2, z, rx, ry)
// with (u, v) the screen mean, (A, B, C) the conic (inverse 2D covariance), k = -log2(e)/2,
// A' = k A, B' = 2 k B, C' = k C, L = log2(aleph), so that log2(aleph K(p)) = L + dx (A' dx + B' dy) + C' dy^2.
// z is the FP32 view depth (the sort key); (rx, ry) are conservative half extents of the bounding box of the
// ellipse where alpha >= alpha_min (0: the splat takes no tile).
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kConicScale = -0.5f * 1.4426950408889634f;

// Per-Gaussian gradient buffer written by the replay (3 float4 per Gaussian): with w = dL/d(log2 alpha) at
// each pixel and (dx, dy) = p - (u, v), the sums over pixels of
//   (w dx, w dy, w dx^2, w dx dy, w dy^2, w, dL/dE0, dL/dE1, dL/dE2, 0, 0, 0),
// the first six divided by ln 2 (the projection backward multiplies it back).
// The record gradient follows: dA' = sum w dx^2, dB' = sum w dx dy, dC' = sum w dy^2, dL = sum w,
// du = -(2A' sum w dx + B' sum w dy), dv = -(B' sum w dx + 2C' sum w dy).

// Per-pixel replay state, 2 float4 per pixel (App. C: E_k is computed in the forward pass and handed
// to the adjoint pass).
//   quadratic:   s0 = (n | sat << 31, E_k), s1 = (A = sum_{i<k} E_i alpha_i, taubar_k)
//   blended:     s0 = (n | sat << 31, E_k), s1 = (sum_{i<k} E_i alpha_i P_i, sum_{i<k} alpha_i P_i)
//   exponential: s0 = (n, C = L0 including background), s1 = (T_end, 0, 0, 0)
//   Vicini:      s0 = (n | linear sat << 31, E_k of the linear list), s1 = (L0 of the exponential list, 0)
// n = number of list entries of the pixel's tile that the forward pass walked through.

// ---- programmatic dependent launch ------------------------------------------------------------------
//
// A kernel started with launch_pdl is scheduled as the CTAs of the kernel before it on the stream exit,
// without waiting for that grid's completion to be processed: its CTAs wait in pdl_wait() until that grid
// has completed and its memory is visible. Every kernel started with launch_pdl calls pdl_wait() before its
// first global memory access; pdl_wait() is a no-op in a kernel started by an ordinary launch. No kernel
// triggers its dependents early (griddepcontrol.launch_dependents): measured on GB300, early triggers made
// the radix passes slower (waiting CTAs of the next kernel on the SMs), and the trigger at exit is what
// shortens the chains of small kernels (depth sort of 0.5M keys 88 -> 64 us, tile sort of 4.2M pairs
// 81 -> 67 us, scan 52 -> 46 us per render).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---- helpers shared bit-for-bit by the forward and the replay kernels ---------------------------

__device__ __forceinline__ float fast_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Approximate reciprocal (PTX rcp.approx, within 1 ulp): only where the value feeds a gradient, never a
// compositing decision.
__device__ __forceinline__ float fast_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// log2 of aleph * K(p) for the splat (r0, r1) at pixel row py, given dx = px - u and adx = A' dx of the
// pixel's column (so pixels of one column share them); FP32, fixed operation order.
__device__ __forceinline__ float splat_log2_alpha_col(float dx, float adx, float py, float4 r0, float4 r1,
                                                      float& dy) {
  dy = __fsub_rn(py, r0.y);
  float t = __fmaf_rn(r0.w, dy, adx);
  float q = __fmaf_rn(dx, t, __fmul_rn(__fmul_rn(r1.x, dy), dy));
  return __fadd_rn(r1.y, q);
}

// log2 of aleph * K(p) for the splat (r0, r1) at pixel centre (px, py); the same arithmetic.
__device__ __forceinline__ float splat_log2_alpha(float px, float py, float4 r0, float4 r1, float& dx, float& dy) {
  dx = __fsub_rn(px, r0.x);
  return splat_log2_alpha_col(dx, __fmul_rn(r0.z, dx), py, r0, r1, dy);
}

// Quadratic slope term alpha (1 + c taubar), clamped at 0 (Table 1 with the [.]_+ of T).
__device__ __forceinline__ float quad_slope(float alpha, float c, float tau) {
  return fmaxf(__fmul_rn(alpha, __fmaf_rn(c, tau, 1.0f)), 0.0f);
}

// Blended slope term alpha (1 - gamma + gamma P), P = prod_{j<i}(1 - alpha_j) (Table 1).
__device__ __forceinline__ float blend_slope(float alpha, float gamma, float one_minus_gamma, float P) {
  return __fmul_rn(alpha, __fmaf_rn(gamma, P, one_minus_gamma));
}

// ---- host-side objects ---------------------------------------------------------------------------

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  template <typename T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

}  // namespace ngs

struct ngs_ctx {
  std::string err;
  int device = 0;
  int num_sms = 0;
  ngs::DevBuf hist;      // radix histograms
  ngs::DevBuf scan_tmp;  // block sums of scans
  ngs::DevBuf grad2d;    // per-Gaussian splat-record gradients (backward)
  ngs::DevBuf total;     // device-side pair count (uint64) and error word (uint64)
  ngs::DevBuf flush;     // autotuner: scratch cleared between timed calls to evict L2
  ngs::DevBuf loss_tmp;  // image loss: moment and partial-derivative planes
  ngs::DevBuf densify_tmp, densify_totals;  // split / prune decisions, scans and totals
  ngs::DevBuf check_word;  // checked mode: one bit per parameter array holding a non-finite value
  bool checked = false;    // checked mode (ngs_set_checked)
  uint64_t* h_total = nullptr;    // pinned, mapped mirror of the scalars read back (kMirrorWords words),
                                  // written by publish_words
  uint64_t* d_h_total = nullptr;  // its device-side address
  bool timing = false;
  struct Pending { cudaEvent_t a, b; int stage; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  double stage_ms[NGS_NUM_STAGES] = {0};
  int64_t stage_launches[NGS_NUM_STAGES] = {0};
  int64_t launches = 0;
  bool graphs = false;                 // capture each render phase once per configuration and replay it
  cudaStream_t cap_stream = nullptr;   // private stream for capturing
  int64_t graph_captures = 0;
};

namespace ngs {
// A captured render phase of a frame, replayed while its launch arguments (`key`) are unchanged.
struct GraphSlot {
  std::vector<uint8_t> key;
  cudaGraphExec_t exec = nullptr;
  int stage_launches[NGS_NUM_STAGES] = {0};
  int g_final = 0, p_final = 0;
};
}  // namespace ngs

struct ngs_frame {
  ngs_ctx* ctx = nullptr;
  bool has_render = false;
  int64_t n = 0;             // Gaussians
  int64_t pairs = 0;
  int n_views = 0;
  int64_t n_pixels = 0;      // all views
  ngs::RenderParams rp;
  std::vector<ngs::ViewParams> view_host;  // the views of the last render (host copy)
  std::vector<int64_t> pix_base;           // [n_views + 1]
  std::vector<uint32_t> tile_base;         // [n_views + 1]
  ngs::ViewParams* h_views = nullptr;      // pinned, mapped staging of the view table
  const uint32_t* d_h_views = nullptr;     // its device-side address
  size_t h_views_cap = 0;
  cudaEvent_t views_uploaded = nullptr;    // recorded after the last upload from h_views
  ngs::DevBuf views;                       // device view table
  ngs::DevBuf rec, tile_count, gkeys[2], gvals[2], offsets;
  ngs::DevBuf ptile[2], pvals[2], ranges, state;
  ngs::DevBuf keys64;  // 64-bit keys, materialised only for ngs_frame_view_get
  ngs::DevBuf work;    // persistent schedule: tiles by descending pair count
  ngs::DevBuf sched;   // persistent schedule: kSchedWords counters (see launch_tile_order)
  ngs::GraphSlot graph[2];  // phase 1 (projection .. pair count) and phase 2 (emission .. composite)
  uint32_t pair_cap = 0;    // pair capacity of the captured phase 2 and of asynchronous renders
  // asynchronous renders (ngs_frame_set_async): a kernel at the end of each one writes its status into a
  // mapped pinned mirror: [0] the largest pair count since the last ngs_frame_status, [1] the error bits
  // since then (kCheck*), [2] the last render's pair count; `done` is recorded after it
  bool async = false;
  bool pending = false;              // an asynchronous render whose status has not been read
  bool last_async = false;           // the last render was asynchronous
  uint64_t* h_status = nullptr;
  uint64_t* d_status = nullptr;
  cudaEvent_t done = nullptr;
  int g_final = 0;  // which gvals[] holds the depth-sorted Gaussian order
  int p_final = 0;  // which ptile[]/pvals[] hold the sorted pairs
};

namespace ngs {

// the render and backward pipelines (api.cu), also used by the autotuner and the server
int render_views(ngs_ctx* ctx, ngs_frame* f, const ngs_gaussians* g, const ngs_camera* cams, int n_views,
                 const ngs_model* model, const ngs_options* o, float* image, int32_t* overdraw, cudaStream_t s);
// Admission of a render's sort buffers: called with stage 0 and the depth-sort bytes before phase 1, and
// with stage 1 and the pair-sort bytes once the exact pair count is known; anything but NGS_OK stops the
// render with that status.
typedef int (*AdmitFn)(void* user, int stage, size_t bytes);
// The same pipeline writing view v's image / overdraw map to images[v] / overdraws[v] ([H][W][3] / [H][W];
// overdraws may be null, or hold nulls).
int render_views_out(ngs_ctx* ctx, ngs_frame* f, const ngs_gaussians* g, const ngs_camera* cams, int n_views,
                     const ngs_model* model, const ngs_options* o, float* const* images, int32_t* const* overdraws,
                     cudaStream_t s, AdmitFn admit = nullptr, void* admit_user = nullptr);
int backward_frame(ngs_ctx* ctx, const ngs_frame* f, const ngs_gaussians* g, const float* dl_dimage,
                   const ngs_grads* out, cudaStream_t s);

// argument checks (api.cu); ctx may be null (no message is kept then)
int check_camera(ngs_ctx* ctx, const ngs_camera* cam);
int check_model(ngs_ctx* ctx, const ngs_model* model);

// error / allocation helpers (api.cu)
int fail(ngs_ctx* ctx, int code, const std::string& msg);
// Device allocation of `bytes` into b, unless it already holds that much; a new allocation takes
// grown_size(current capacity, bytes): at least a quarter more than before, rounded up to 256 B.
int ensure(ngs_ctx* ctx, DevBuf& b, size_t bytes);
size_t grown_size(size_t cap, size_t bytes);
// Slots of the context's mapped mirror: the pair count and the device error word of the last render, the
// loss sums (two doubles), the densified Gaussian count, the checked-mode scan's bits.
constexpr int kMirrorTotal = 0, kMirrorLoss = 2, kMirrorDensify = 4, kMirrorChecked = 5, kMirrorWords = 8;
// Copy n (<= 32) 64-bit device words into mirror slots [slot, slot + n) with one kernel on stream s.
void publish_words(ngs_ctx* ctx, const uint64_t* src, int n, int slot, cudaStream_t s);
void stage_begin(ngs_ctx* ctx, cudaStream_t s, int stage, cudaEvent_t* out);
void stage_end(ngs_ctx* ctx, cudaStream_t s, int stage, cudaEvent_t start, int launches);

// kernels' host launchers
// For every view v and Gaussian i, record r = v n + i: splat record, depth key (0xFFFFFFFF for splats
// without tiles), tile count and order[r] = r.
// cam0: the camera of view 0 (used when rp.n_views == 1).
void launch_project(const ngs_gaussians& g, const ViewParams* views, const CamParams& cam0, const RenderParams& rp,
                    float4* rec, uint32_t* depth_key, uint32_t* tile_count, uint32_t* order, cudaStream_t s);
// Gradients w.r.t. the Gaussian parameters, summed over the views.
// cam0: the camera of view 0 (the only one when rp.n_views == 1).
void launch_project_backward(const ngs_gaussians& g, const ViewParams* views, const CamParams& cam0,
                             const RenderParams& rp, const uint32_t* tile_count, const float4* grad2d,
                             const ngs_grads& out, int num_sms, cudaStream_t s);
// Stable radix sort of (key, value) pairs on bits [begin_bit, end_bit), independently within each of
// `nseg` segments of seg_len items. If n_dev is not null, only the first min(*n_dev, seg_len) items of a
// segment are sorted (a count known on the device only; seg_len is then the capacity). Returns the index
// (0/1) of the buffer pair holding the result; launches counted into *launches.
int radix_sort_u32(uint32_t* keys[2], uint32_t* vals[2], uint32_t seg_len, uint32_t nseg, const uint32_t* n_dev,
                   int begin_bit, int end_bit, uint32_t* hist, cudaStream_t s, int* launches);
size_t radix_hist_words(uint32_t seg_len, uint32_t nseg);
// exclusive scan of tile_count[order[i]] into offsets[0..n] (offsets[n] = total) and the total into
// *total (uint64, device); returns the error of its own runtime calls (n = 0 clears both with memsets)
cudaError_t launch_scan_counts(const uint32_t* tile_count, const uint32_t* order, uint32_t n, uint32_t* offsets,
                               uint64_t* block_sums, uint64_t* total, cudaStream_t s, int* launches);
size_t scan_tmp_words(uint32_t n);
// One (view-local tile, record index) pair per covered tile, in the order of `order` (n_records entries):
// the records are in (view, depth) order, so sorting the pairs stably by the local tile alone orders them by
// (local tile, view, depth): every (view, tile) list is contiguous and in the order of the 64-bit keys
// (global tile << 32 | depth bits).
// Pairs at slots >= cap are not written (an asynchronous render whose count exceeds its capacity).
void launch_emit_pairs(const float4* rec, const uint32_t* order, const uint32_t* offsets, const ViewParams* views,
                       const RenderParams& rp, uint32_t* tiles, uint32_t* vals, uint32_t cap, cudaStream_t s);
// keys[i] = global tile of pair i << 32 | bits(depth of record vals[i]) (diagnostics).
void launch_compose_keys(const uint32_t* tiles, const uint32_t* vals, const float4* rec, const ViewParams* views,
                         uint32_t n_per_view, uint32_t n_views, uint32_t npairs, uint64_t* keys, cudaStream_t s);
// [start, end) of every global tile's pairs into `ranges`, which the caller has zeroed (zero-length ranges
// stay (0, 0)); npairs_cap items are covered by the grid, of which the first *npairs_dev are valid if
// npairs_dev is not null. A pair naming a record or tile out of range is skipped and reported in *check.
void launch_tile_ranges(const uint32_t* tiles, const uint32_t* vals, const ViewParams* views, uint32_t n_per_view,
                        uint32_t n_views, uint32_t npairs_cap, const uint32_t* npairs_dev, uint32_t ntiles,
                        uint2* ranges, uint32_t* check, cudaStream_t s);
// Persistent schedule: work[] lists all tiles by descending pair count (buckets of floor(log2(pairs)),
// any order within a bucket). `sched` holds kSchedWords zeroed words: [0] forward and [1] backward work
// counters, then per-bucket counts and cursors.
constexpr int kCostBuckets = 33;
constexpr int kSchedWords = 2 + 2 * kCostBuckets;
void launch_tile_order(const uint2* ranges, uint32_t ntiles, uint32_t* sched, uint32_t* work, cudaStream_t s,
                       int* launches);
// Composite launches. work/counter null: one CTA per tile; else persistent CTAs (num_sms x occupancy)
// taking tiles from work[] through the zeroed counter.
void launch_composite_forward(const float4* rec, const uint32_t* ids, const uint2* ranges, const RenderParams& rp,
                              const ViewParams* views, float* image, int32_t* overdraw, float4* state,
                              const uint32_t* work, uint32_t* counter, int num_sms, cudaStream_t s);
void launch_composite_backward(const float4* rec, const uint32_t* ids, const uint2* ranges, const RenderParams& rp,
                               const ViewParams* views, const float* dl_dimage, const float4* state, float4* grad2d,
                               const uint32_t* work, uint32_t* counter, int num_sms, cudaStream_t s);

}  // namespace ngs
