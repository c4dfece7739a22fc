// C ABI of the ngs library: contexts, frames, argument checks, buffer management and the render /
// backward pipelines (projection -> depth sort -> scan + key emission -> tile sort -> tile ranges ->
// composite; composite replay -> projection backward).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "ngs_internal.cuh"

namespace ngs {

int fail(ngs_ctx* ctx, int code, const std::string& msg) {  // ctx may be null
  if (ctx) ctx->err = msg;
  return code;
}

size_t grown_size(size_t cap, size_t bytes) {
  if (cap && bytes <= cap) return cap;
  const size_t nb = std::max(bytes, cap + cap / 4);
  return (std::max<size_t>(nb, 256) + 255) & ~(size_t)255;
}

int ensure(ngs_ctx* ctx, DevBuf& b, size_t bytes) {
  if (bytes <= b.cap && b.p) return NGS_OK;
  const size_t nb = grown_size(b.p ? b.cap : 0, bytes);
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  cudaError_t e = cudaMalloc(&b.p, nb);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    char msg[160];
    snprintf(msg, sizeof msg, "device allocation of %zu bytes failed: %s", nb, cudaGetErrorString(e));
    return fail(ctx, NGS_ERR_OUT_OF_MEMORY, msg);
  }
  b.cap = nb;
  return NGS_OK;
}

static cudaEvent_t take_event(ngs_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void stage_begin(ngs_ctx* ctx, cudaStream_t s, int, cudaEvent_t* out) {
  *out = nullptr;
  if (!ctx->timing) return;
  *out = take_event(ctx);
  cudaEventRecord(*out, s);
}

void stage_end(ngs_ctx* ctx, cudaStream_t s, int stage, cudaEvent_t start, int launches) {
  ctx->launches += launches;
  ctx->stage_launches[stage] += launches;
  if (!ctx->timing || !start) return;
  cudaEvent_t b = take_event(ctx);
  cudaEventRecord(b, s);
  ctx->pending.push_back({start, b, stage});
}

// Host <-> device traffic of a render without the copy engines: a render would otherwise wait for its
// view table and its pair count behind whatever bulk copies other streams have queued on the engines.
// The view table is read by a kernel from mapped pinned memory over the host link...
__global__ void copy_words_kernel(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, uint32_t n) {
  pdl_wait();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i];
}

// ... and the scalars the host reads back (the pair count and the error word, loss sums, a densified count)
// are written by a kernel into the context's mapped pinned mirror, read after synchronising with the stream.
__global__ void publish_words_kernel(const uint64_t* __restrict__ src, uint64_t* dst, int n) {
  pdl_wait();
  if ((int)threadIdx.x < n) dst[threadIdx.x] = src[threadIdx.x];
  __threadfence_system();
}

// End of an asynchronous render: folds its pair count and error bits into the frame's mapped status
// (the capacity bit when the count exceeded `cap`) and clears the context's error word for the next render.
// One thread: the status words are read, modified and written in host memory.
__global__ void finish_async_kernel(uint64_t* total, uint64_t* status, uint32_t cap) {
  pdl_wait();
  if (threadIdx.x != 0) return;
  const uint64_t count = total[0];
  const uint64_t err = total[1] | (count > cap ? (uint64_t)kCheckCapacity : 0ull);
  status[0] = count > status[0] ? count : status[0];
  status[1] |= err;
  status[2] = count;
  total[1] = 0;
  __threadfence_system();
}

void publish_words(ngs_ctx* ctx, const uint64_t* src, int n, int slot, cudaStream_t s) {
  launch_pdl(publish_words_kernel, 1, 32, 0, s, src, ctx->d_h_total + slot, n);
}

static void free_buf(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

static int check_launch(ngs_ctx* ctx, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    char msg[200];
    snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
    return fail(ctx, NGS_ERR_CUDA, msg);
  }
  return NGS_OK;
}

constexpr int kMaxViews = 4096;

static int tile_bits(uint32_t ntiles) {
  int b = 0;
  while (b < 32 && (1ull << b) < ntiles) ++b;
  return b;
}

}  // namespace ngs

using namespace ngs;

#define NGS_TRY(x)             \
  do {                         \
    int _rc = (x);             \
    if (_rc != NGS_OK) return _rc; \
  } while (0)

int ngs::check_camera(ngs_ctx* ctx, const ngs_camera* cam) {
  if (!cam) return fail(ctx, NGS_ERR_INVALID_ARG, "null camera");
  if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384)
    return fail(ctx, NGS_ERR_INVALID_ARG, "image size out of range 1..16384");
  if (!(cam->fx > 0) || !(cam->fy > 0) || !isfinite(cam->cx) || !isfinite(cam->cy))
    return fail(ctx, NGS_ERR_INVALID_ARG, "invalid intrinsics");
  for (int i = 0; i < 12; ++i)
    if (!isfinite(cam->viewmat[i])) return fail(ctx, NGS_ERR_INVALID_ARG, "non-finite view matrix");
  return NGS_OK;
}

int ngs::check_model(ngs_ctx* ctx, const ngs_model* model) {
  if (!model) return fail(ctx, NGS_ERR_INVALID_ARG, "null model");
  if (model->kind == NGS_MODEL_QUAD) {
    if (!(model->param >= -0.5f) || !isfinite(model->param))
      return fail(ctx, NGS_ERR_INVALID_ARG, "quadratic model needs c >= -0.5");
  } else if (model->kind == NGS_MODEL_BLEND || model->kind == NGS_MODEL_VICINI) {
    if (!(model->param >= 0.f && model->param <= 1.f))
      return fail(ctx, NGS_ERR_INVALID_ARG, "blended / Vicini model needs gamma in [0, 1]");
  } else if (model->kind != NGS_MODEL_EXP) {
    return fail(ctx, NGS_ERR_INVALID_ARG, "unknown transmittance model");
  }
  return NGS_OK;
}

static int check_inputs(ngs_ctx* ctx, const ngs_gaussians* g, const ngs_model* model, const ngs_options* o) {
  if (!g || !model || !o) return fail(ctx, NGS_ERR_INVALID_ARG, "null argument");
  if (g->n < 0 || g->n >= (1ll << 31)) return fail(ctx, NGS_ERR_INVALID_ARG, "n out of range [0, 2^31)");
  if (g->sh_degree < 0 || g->sh_degree > 3) return fail(ctx, NGS_ERR_INVALID_ARG, "sh_degree must be 0..3");
  if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh))
    return fail(ctx, NGS_ERR_INVALID_ARG, "null Gaussian parameter array");
  NGS_TRY(check_model(ctx, model));
  bool tile_ok = (o->tile_w == 8 && o->tile_h == 8) || (o->tile_w == 16 && o->tile_h == 16) ||
                 (o->tile_w == 16 && o->tile_h == 32);
  if (!tile_ok) return fail(ctx, NGS_ERR_INVALID_ARG, "tile shape must be 8x8, 16x16 or 16x32");
  if (!(o->alpha_min > 0.f && o->alpha_min < 1.f) || !(o->alpha_max > o->alpha_min && o->alpha_max <= 1.f))
    return fail(ctx, NGS_ERR_INVALID_ARG, "need 0 < alpha_min < alpha_max <= 1");
  if (!(o->t_eps >= 0.f && o->t_eps < 1.f) || !(o->dilation >= 0.f) || !(o->near_plane > 0.f) ||
      o->max_splats < 0)
    return fail(ctx, NGS_ERR_INVALID_ARG, "invalid option value");
  const int P = o->tile_w * o->tile_h;
  if (o->chunk != 0 && o->chunk != P / 2 && o->chunk != P && o->chunk != 2 * P)
    return fail(ctx, NGS_ERR_INVALID_ARG, "chunk must be 0 or half, once or twice the tile's pixel count");
  if (o->schedule != NGS_SCHEDULE_TILES && o->schedule != NGS_SCHEDULE_PERSISTENT)
    return fail(ctx, NGS_ERR_INVALID_ARG, "unknown schedule");
  for (int i = 0; i < 3; ++i)
    if (!isfinite(o->background[i])) return fail(ctx, NGS_ERR_INVALID_ARG, "non-finite background");
  return NGS_OK;
}

static void camera_params(const ngs_camera* cam, CamParams& cp) {
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) cp.R[3 * r + c] = cam->viewmat[4 * r + c];
    cp.t[r] = cam->viewmat[4 * r + 3];
  }
  for (int c = 0; c < 3; ++c)
    cp.campos[c] = -(cp.R[c] * cp.t[0] + cp.R[3 + c] * cp.t[1] + cp.R[6 + c] * cp.t[2]);
  cp.fx = cam->fx;
  cp.fy = cam->fy;
  cp.cx = cam->cx;
  cp.cy = cam->cy;
  cp.W = cam->width;
  cp.H = cam->height;
}

// Bytes of every device buffer a render (and its backward) asks for: the one place these sizes are
// written, used by the render itself and by ngs_workspace_bytes. cap: the pair buffers' item count.
struct BufferPlan {
  size_t rec, tile_count, keys, vals, offsets, ranges, state, views, work, sched;  // frame, per render
  size_t pair_tile, pair_val;                                                       // frame, per pair
  size_t scan_tmp, total, hist1, hist2;                                             // context
  size_t grad2d;                                                                    // context, backward
};

static BufferPlan plan_buffers(uint64_t R, uint32_t n, uint32_t n_views, uint64_t ntiles, uint64_t pix_total,
                               int schedule, uint64_t cap) {
  BufferPlan b;
  const size_t r1 = (size_t)std::max<uint64_t>(R, 1);
  b.rec = sizeof(float4) * 3 * r1;
  b.tile_count = b.keys = b.vals = sizeof(uint32_t) * r1;
  b.offsets = sizeof(uint32_t) * ((size_t)R + 1);
  b.ranges = sizeof(uint2) * (size_t)ntiles;
  b.state = sizeof(float4) * 2 * (size_t)pix_total;
  b.views = sizeof(ViewParams) * (size_t)n_views;
  b.work = schedule == NGS_SCHEDULE_PERSISTENT ? sizeof(uint32_t) * (size_t)std::max<uint64_t>(ntiles, 1) : 0;
  b.sched = schedule == NGS_SCHEDULE_PERSISTENT ? sizeof(uint32_t) * kSchedWords : 0;
  b.pair_tile = b.pair_val = sizeof(uint32_t) * (size_t)std::max<uint64_t>(cap, 1);
  b.scan_tmp = sizeof(uint64_t) * scan_tmp_words((uint32_t)R);
  b.total = 2 * sizeof(uint64_t);
  b.hist1 = sizeof(uint32_t) * radix_hist_words(std::max(n, 1u), std::max(n_views, 1u));
  b.hist2 = sizeof(uint32_t) * radix_hist_words((uint32_t)std::max<uint64_t>(cap, 1), 1);
  b.grad2d = sizeof(float4) * 3 * r1;
  return b;
}

// Stage the view table in the frame's pinned buffer (the copy to the device is a launch of phase 1). The
// staging is rewritten only after the previous copy from it has completed.
static int stage_views(ngs_ctx* ctx, ngs_frame* f) {
  size_t bytes = sizeof(ViewParams) * f->view_host.size();
  if (f->views_uploaded) {
    cudaError_t e = cudaEventSynchronize(f->views_uploaded);
    if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("view table upload: ") + cudaGetErrorString(e));
  } else if (cudaEventCreateWithFlags(&f->views_uploaded, cudaEventDisableTiming) != cudaSuccess) {
    f->views_uploaded = nullptr;
    return fail(ctx, NGS_ERR_CUDA, "cudaEventCreate failed");
  }
  if (f->h_views_cap < f->view_host.size()) {
    if (f->h_views) cudaFreeHost(f->h_views);
    f->h_views = nullptr;
    f->h_views_cap = 0;
    void* dev_alias = nullptr;
    if (cudaHostAlloc((void**)&f->h_views, bytes, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(&dev_alias, f->h_views, 0) != cudaSuccess) {
      cudaGetLastError();
      if (f->h_views) cudaFreeHost(f->h_views);
      f->h_views = nullptr;
      return fail(ctx, NGS_ERR_OUT_OF_MEMORY, "mapped pinned allocation of the view table failed");
    }
    f->d_h_views = static_cast<const uint32_t*>(dev_alias);
    f->h_views_cap = f->view_host.size();
  }
  NGS_TRY(ensure(ctx, f->views, plan_buffers(0, 0, (uint32_t)f->view_host.size(), 0, 0, 0, 0).views));
  memcpy(f->h_views, f->view_host.data(), bytes);
  return NGS_OK;
}

// The bytes ngs_workspace_bytes reports, from one plan: a fresh allocation of each buffer.
static size_t fresh_bytes(size_t bytes) { return bytes ? grown_size(0, bytes) : (size_t)0; }
static size_t plan_frame_fixed(const BufferPlan& b) {
  return fresh_bytes(b.rec) + fresh_bytes(b.tile_count) + 2 * fresh_bytes(b.keys) + 2 * fresh_bytes(b.vals) +
         fresh_bytes(b.offsets) + fresh_bytes(b.ranges) + fresh_bytes(b.state) + fresh_bytes(b.views) +
         fresh_bytes(b.work) + fresh_bytes(b.sched);
}
static size_t plan_frame_pairs(const BufferPlan& b) { return 2 * fresh_bytes(b.pair_tile) + 2 * fresh_bytes(b.pair_val); }
static size_t plan_context(const BufferPlan& b) {
  return fresh_bytes(b.scan_tmp) + fresh_bytes(b.total) + grown_size(grown_size(0, b.hist1), b.hist2);
}

// Checked mode: every parameter of the Gaussians finite, else NGS_ERR_INVALID_ARG naming the array.
__global__ void nonfinite_kernel(const float* __restrict__ a, size_t count, uint32_t bit, uint32_t* flag) {
  pdl_wait();
  bool bad = false;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(a[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, bit);
}

static int check_finite(ngs_ctx* ctx, const ngs_gaussians* g, cudaStream_t s) {
  if (g->n == 0) return NGS_OK;
  NGS_TRY(ensure(ctx, ctx->check_word, sizeof(uint64_t)));
  cudaError_t e = cudaMemsetAsync(ctx->check_word.p, 0, sizeof(uint64_t), s);
  if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("checked mode: ") + cudaGetErrorString(e));
  const size_t n = (size_t)g->n, K3 = 3 * (size_t)(g->sh_degree + 1) * (size_t)(g->sh_degree + 1);
  const float* arrays[5] = {g->means, g->log_scales, g->quats, g->opacity_logits, g->sh};
  const size_t counts[5] = {3 * n, 3 * n, 4 * n, n, K3 * n};
  for (int k = 0; k < 5; ++k) {
    const unsigned blocks = (unsigned)std::min<size_t>((counts[k] + 255) / 256, (size_t)ctx->num_sms * 8);
    launch_pdl(nonfinite_kernel, blocks, 256, 0, s, arrays[k], counts[k], 1u << k, ctx->check_word.as<uint32_t>());
  }
  publish_words(ctx, ctx->check_word.as<uint64_t>(), 1, kMirrorChecked, s);
  ctx->launches += 6;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("checked mode: ") + cudaGetErrorString(e));
  const uint64_t bits = static_cast<volatile uint64_t*>(ctx->h_total)[kMirrorChecked];
  static const char* names[5] = {"means", "log_scales", "quats", "opacity_logits", "sh"};
  for (int k = 0; k < 5; ++k)
    if (bits & (1u << k))
      return fail(ctx, NGS_ERR_INVALID_ARG, std::string("checked mode: non-finite value in ") + names[k]);
  return NGS_OK;
}

// Everything a render derives from its arguments before the first launch.
struct RenderPlan {
  RenderParams rp;
  const ngs_gaussians* g;
  uint32_t n, R, ntiles;
  uint64_t pix_total;
  float* image;
  int32_t* overdraw;
};

// Phase 1: view table upload, projection, depth sort, scan of the tile counts, and the pair count (and the
// device error word) written into the context's mapped pinned mirror. Launches only.
static cudaError_t phase1(ngs_ctx* ctx, ngs_frame* f, const RenderPlan& pl, cudaStream_t s) {
  const RenderParams& rp = pl.rp;
  const ViewParams* views = f->views.as<ViewParams>();
  cudaEvent_t ev;
  // 1. the view table to the device; projection of every (view, Gaussian): splat records, FP32 depth keys
  //    (all-ones for splats that take no tile), tile counts
  stage_begin(ctx, s, 0, &ev);
  {
    static_assert(sizeof(ViewParams) % 4 == 0, "the view table is copied in 4-byte words");
    const uint32_t words = (uint32_t)(sizeof(ViewParams) * f->view_host.size() / 4);
    launch_pdl(copy_words_kernel, std::min((words + 255) / 256, 64u), 256, 0, s, f->d_h_views, f->views.as<uint32_t>(),
               words);
  }
  launch_project(*pl.g, views, f->view_host[0].cam, rp, f->rec.as<float4>(), f->gkeys[0].as<uint32_t>(),
                 f->tile_count.as<uint32_t>(), f->gvals[0].as<uint32_t>(), s);
  stage_end(ctx, s, 0, ev, pl.n ? 2 : 1);
  // 2. stable sort of each view's splats by FP32 depth (ties keep Gaussian order)
  stage_begin(ctx, s, 1, &ev);
  int launches = 0;
  {
    uint32_t* k2[2] = {f->gkeys[0].as<uint32_t>(), f->gkeys[1].as<uint32_t>()};
    uint32_t* v2[2] = {f->gvals[0].as<uint32_t>(), f->gvals[1].as<uint32_t>()};
    f->g_final = radix_sort_u32(k2, v2, pl.n, rp.n_views, nullptr, 0, 32, ctx->hist.as<uint32_t>(), s, &launches);
  }
  stage_end(ctx, s, 1, ev, launches);
  // 3. exclusive scan of the tile counts in (view, depth) order; the pair count goes to the host mirror
  stage_begin(ctx, s, 2, &ev);
  launches = 0;
  const cudaError_t e = launch_scan_counts(f->tile_count.as<uint32_t>(), f->gvals[f->g_final].as<uint32_t>(), pl.R,
                                           f->offsets.as<uint32_t>(), ctx->scan_tmp.as<uint64_t>(),
                                           ctx->total.as<uint64_t>(), s, &launches);
  publish_words(ctx, ctx->total.as<uint64_t>(), 2, kMirrorTotal, s);
  stage_end(ctx, s, 2, ev, launches + 1);
  return e;
}

// Phase 2: key emission, tile sort, tile ranges (+ work list), composite. `cap` items are covered by the
// sort's grid; with np_dev (graph replays) the kernels read the actual pair count from the device.
static cudaError_t phase2(ngs_ctx* ctx, ngs_frame* f, const RenderPlan& pl, uint32_t cap, const uint32_t* np_dev,
                          bool async, cudaStream_t s) {
  const RenderParams& rp = pl.rp;
  const ViewParams* views = f->views.as<ViewParams>();
  cudaEvent_t ev;
  // zeroing first, so that the kernels from the emission to the composite follow one another directly
  // (programmatic dependent launches)
  cudaError_t e = cudaMemsetAsync(f->ranges.p, 0, sizeof(uint2) * (size_t)pl.ntiles, s);
  if (e == cudaSuccess && rp.schedule == NGS_SCHEDULE_PERSISTENT)
    e = cudaMemsetAsync(f->sched.p, 0, sizeof(uint32_t) * kSchedWords, s);
  if (e != cudaSuccess) return e;
  stage_begin(ctx, s, 2, &ev);
  launch_emit_pairs(f->rec.as<float4>(), f->gvals[f->g_final].as<uint32_t>(), f->offsets.as<uint32_t>(), views, rp,
                    f->ptile[0].as<uint32_t>(), f->pvals[0].as<uint32_t>(), cap, s);
  stage_end(ctx, s, 2, ev, pl.R ? 1 : 0);
  // 4. stable sort of the pairs by view-local tile: the (view, depth) order inside each local tile is kept,
  //    so every (view, tile) list is contiguous and in the order of the 64-bit (tile << 32 | depth) keys
  stage_begin(ctx, s, 3, &ev);
  int launches = 0;
  {
    uint32_t* k2[2] = {f->ptile[0].as<uint32_t>(), f->ptile[1].as<uint32_t>()};
    uint32_t* v2[2] = {f->pvals[0].as<uint32_t>(), f->pvals[1].as<uint32_t>()};
    int max_tiles = 0;  // the pairs carry view-local tiles
    for (const ViewParams& vp : f->view_host) max_tiles = std::max(max_tiles, vp.tiles_x * vp.tiles_y);
    f->p_final = radix_sort_u32(k2, v2, cap, 1, np_dev, 0, tile_bits((uint32_t)max_tiles), ctx->hist.as<uint32_t>(), s,
                                &launches);
  }
  stage_end(ctx, s, 3, ev, launches);
  // 5. per-tile [start, end); for the persistent schedule, the tiles by descending pair count
  stage_begin(ctx, s, 4, &ev);
  launches = cap ? 1 : 0;
  launch_tile_ranges(f->ptile[f->p_final].as<uint32_t>(), f->pvals[f->p_final].as<uint32_t>(), views, pl.n, rp.n_views,
                     cap, np_dev, pl.ntiles, f->ranges.as<uint2>(), rp.check, s);
  const uint32_t* work = nullptr;
  uint32_t* counter = nullptr;
  if (rp.schedule == NGS_SCHEDULE_PERSISTENT) {
    launch_tile_order(f->ranges.as<uint2>(), pl.ntiles, f->sched.as<uint32_t>(), f->work.as<uint32_t>(), s,
                      &launches);
    work = f->work.as<uint32_t>();
    counter = f->sched.as<uint32_t>();
  }
  stage_end(ctx, s, 4, ev, launches);
  // 6. composite every tile of every view
  stage_begin(ctx, s, 5, &ev);
  launch_composite_forward(f->rec.as<float4>(), f->pvals[f->p_final].as<uint32_t>(), f->ranges.as<uint2>(), rp, views,
                           pl.image, pl.overdraw, f->state.as<float4>(), work, counter, ctx->num_sms, s);
  stage_end(ctx, s, 5, ev, 1);
  if (async) {
    launch_pdl(finish_async_kernel, 1, 32, 0, s, ctx->total.as<uint64_t>(), f->d_status, cap);
    ctx->launches += 1;
  }
  return cudaSuccess;
}

// Serialised launch arguments of a phase: a captured graph is replayed only while they are unchanged.
struct KeyBuf {
  std::vector<uint8_t> b;
  template <typename T>
  void add(const T& v) {
    const uint8_t* p = reinterpret_cast<const uint8_t*>(&v);
    b.insert(b.end(), p, p + sizeof(T));
  }
};

// Run one phase: directly, or (graphs enabled) by replaying the frame's graph for it, captured anew on
// the context's capture stream when the key changed.
template <typename Fn>
static int run_phase(ngs_ctx* ctx, ngs_frame* f, int which, const KeyBuf& key, cudaStream_t s, Fn&& launch) {
  const char* what = which == 0 ? "render phase 1" : "render phase 2";
  if (!ctx->graphs) {
    cudaError_t e = launch(s);
    if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return check_launch(ctx, what);
  }
  GraphSlot& g = f->graph[which];
  if (!g.exec || g.key != key.b) {
    if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail(ctx, NGS_ERR_CUDA, "creating the capture stream failed");
    const bool timing = ctx->timing;
    int64_t before[NGS_NUM_STAGES];
    for (int i = 0; i < NGS_NUM_STAGES; ++i) before[i] = ctx->stage_launches[i];
    const int64_t total_before = ctx->launches;
    ctx->timing = false;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t le = launch(ctx->cap_stream);
      e = cudaStreamEndCapture(ctx->cap_stream, &graph);
      if (le != cudaSuccess) e = le;
    }
    ctx->timing = timing;
    for (int i = 0; i < NGS_NUM_STAGES; ++i) {  // counted per replay below, not at capture
      g.stage_launches[i] = (int)(ctx->stage_launches[i] - before[i]);
      ctx->stage_launches[i] = before[i];
    }
    ctx->launches = total_before;
    if (e == cudaSuccess && g.exec) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(g.exec, graph, &info) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
      }
    }
    if (e == cudaSuccess && !g.exec) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g.exec = nullptr;
      g.key.clear();
      return fail(ctx, NGS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    g.key = key.b;
    g.p_final = f->p_final;
    g.g_final = f->g_final;
    ++ctx->graph_captures;
  }
  f->p_final = g.p_final;
  f->g_final = g.g_final;
  cudaError_t e = cudaGraphLaunch(g.exec, s);
  if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  for (int i = 0; i < NGS_NUM_STAGES; ++i) {
    ctx->stage_launches[i] += g.stage_launches[i];
    ctx->launches += g.stage_launches[i];
  }
  return NGS_OK;
}

// The render pipeline for n_views cameras of one set of Gaussians (n_views = 1 for ngs_render).
int ngs::render_views(ngs_ctx* ctx, ngs_frame* f, const ngs_gaussians* g, const ngs_camera* cams, int n_views,
                      const ngs_model* model, const ngs_options* o, float* image, int32_t* overdraw,
                      cudaStream_t s) {
  if (!cams) return fail(ctx, NGS_ERR_INVALID_ARG, "null camera");
  if (n_views < 1 || n_views > kMaxViews) return fail(ctx, NGS_ERR_INVALID_ARG, "n_views out of range 1..4096");
  if (!image) return fail(ctx, NGS_ERR_INVALID_ARG, "null image");
  std::vector<float*> images(n_views);
  std::vector<int32_t*> ods(n_views);
  uint64_t base = 0;
  for (int v = 0; v < n_views; ++v) {  // the packed layout: view v after views 0..v-1
    images[v] = image + 3 * base;
    ods[v] = overdraw ? overdraw + base : nullptr;
    base += (uint64_t)std::max(cams[v].width, 0) * (uint64_t)std::max(cams[v].height, 0);
  }
  return render_views_out(ctx, f, g, cams, n_views, model, o, images.data(), ods.data(), s);
}

int ngs::render_views_out(ngs_ctx* ctx, ngs_frame* f, const ngs_gaussians* g, const ngs_camera* cams, int n_views,
                          const ngs_model* model, const ngs_options* o, float* const* images,
                          int32_t* const* overdraws, cudaStream_t s, AdmitFn admit, void* admit_user) {
  if (!f || f->ctx != ctx) return fail(ctx, NGS_ERR_INVALID_ARG, "frame missing or from another context");
  NGS_TRY(check_inputs(ctx, g, model, o));
  if (!cams || !images) return fail(ctx, NGS_ERR_INVALID_ARG, "null camera or image array");
  if (n_views < 1 || n_views > kMaxViews) return fail(ctx, NGS_ERR_INVALID_ARG, "n_views out of range 1..4096");
  for (int v = 0; v < n_views; ++v) {
    NGS_TRY(check_camera(ctx, &cams[v]));
    if (!images[v]) return fail(ctx, NGS_ERR_INVALID_ARG, "null image");
  }
  f->has_render = false;

  // views, packed: tiles and pixels of view v follow those of views 0..v-1
  f->view_host.resize(n_views);
  f->pix_base.assign(n_views + 1, 0);
  f->tile_base.assign(n_views + 1, 0);
  uint64_t tiles_total = 0, pix_total = 0;
  for (int v = 0; v < n_views; ++v) {
    ViewParams& vp = f->view_host[v];
    memset(&vp, 0, sizeof vp);
    camera_params(&cams[v], vp.cam);
    vp.tiles_x = (cams[v].width + o->tile_w - 1) / o->tile_w;
    vp.tiles_y = (cams[v].height + o->tile_h - 1) / o->tile_h;
    vp.tile_base = (uint32_t)tiles_total;
    vp.pix_base = pix_total;
    vp.image = images[v];
    vp.overdraw = overdraws ? overdraws[v] : nullptr;
    f->tile_base[v] = (uint32_t)tiles_total;
    f->pix_base[v] = (int64_t)pix_total;
    tiles_total += (uint64_t)vp.tiles_x * vp.tiles_y;
    pix_total += (uint64_t)cams[v].width * cams[v].height;
    if (tiles_total >= (1ull << 31)) return fail(ctx, NGS_ERR_INVALID_ARG, "more than 2^31 tiles in the batch");
  }
  f->tile_base[n_views] = (uint32_t)tiles_total;
  f->pix_base[n_views] = (int64_t)pix_total;
  const uint64_t records64 = (uint64_t)g->n * (uint64_t)n_views;
  if (records64 >= (1ull << 32)) return fail(ctx, NGS_ERR_INVALID_ARG, "n * n_views must be below 2^32");

  RenderPlan pl;
  RenderParams& rp = pl.rp;
  memset(&rp, 0, sizeof rp);
  rp.alpha_min = o->alpha_min;
  rp.alpha_max = o->alpha_max;
  rp.t_eps = o->t_eps;
  rp.dilation = o->dilation;
  rp.near_plane = o->near_plane;
  rp.log2_alpha_min = log2f(o->alpha_min);
  for (int c = 0; c < 3; ++c) rp.bg[c] = o->background[c];
  rp.c = model->kind == NGS_MODEL_EXP ? 0.f : model->param;
  rp.c1 = 1.0f - rp.c;
  rp.kind = model->kind;
  rp.tile_w = o->tile_w;
  rp.tile_h = o->tile_h;
  rp.tiles_x = f->view_host[0].tiles_x;
  rp.tiles_y = f->view_host[0].tiles_y;
  rp.width = cams[0].width;
  rp.height = cams[0].height;
  rp.max_splats = o->max_splats;
  rp.chunk = o->chunk ? o->chunk : o->tile_w * o->tile_h;
  rp.schedule = o->schedule;
  rp.sh_degree = g->sh_degree;
  rp.n_gaussians = (uint32_t)g->n;
  rp.n_views = (uint32_t)n_views;
  rp.n_records = (uint32_t)records64;
  rp.n_tiles = (uint32_t)tiles_total;
  // a captured projection takes every camera from the view table, so that a replay serves any pose
  rp.cam_from_table = (n_views > 1 || ctx->graphs) ? 1 : 0;
  pl.g = g;
  pl.n = (uint32_t)g->n;
  pl.R = rp.n_records;
  pl.ntiles = rp.n_tiles;
  pl.pix_total = pix_total;
  pl.image = images[0];
  pl.overdraw = overdraws ? overdraws[0] : nullptr;
  const uint32_t R = pl.R;

  if (ctx->checked) NGS_TRY(check_finite(ctx, g, s));

  // phase 1 buffers (sizes shared with ngs_workspace_bytes)
  const BufferPlan bp = plan_buffers(R, pl.n, (uint32_t)n_views, pl.ntiles, pix_total, rp.schedule, 0);
  NGS_TRY(ensure(ctx, f->rec, bp.rec));
  NGS_TRY(ensure(ctx, f->tile_count, bp.tile_count));
  for (int k = 0; k < 2; ++k) {
    NGS_TRY(ensure(ctx, f->gkeys[k], bp.keys));
    NGS_TRY(ensure(ctx, f->gvals[k], bp.vals));
  }
  NGS_TRY(ensure(ctx, f->offsets, bp.offsets));
  NGS_TRY(ensure(ctx, f->ranges, bp.ranges));
  NGS_TRY(ensure(ctx, f->state, bp.state));
  NGS_TRY(ensure(ctx, ctx->scan_tmp, bp.scan_tmp));
  if (!ctx->total.p) {
    NGS_TRY(ensure(ctx, ctx->total, bp.total));
    const cudaError_t ze = cudaMemsetAsync(ctx->total.p, 0, 2 * sizeof(uint64_t), s);
    if (ze != cudaSuccess) {
      free_buf(ctx->total);  // zeroed on the next render's first use again
      return fail(ctx, NGS_ERR_CUDA, std::string("clearing the pair count: ") + cudaGetErrorString(ze));
    }
  }
  rp.check = reinterpret_cast<uint32_t*>(ctx->total.as<uint64_t>() + 1);
  NGS_TRY(ensure(ctx, ctx->hist, bp.hist1));
  if (rp.schedule == NGS_SCHEDULE_PERSISTENT) {
    NGS_TRY(ensure(ctx, f->work, bp.work));
    NGS_TRY(ensure(ctx, f->sched, bp.sched));
  }
  NGS_TRY(stage_views(ctx, f));
  // admission reserves what ngs_workspace_bytes reports: the frame's record, tile and pixel buffers and the
  // context's scratch now, the pair buffers once the pair count is known
  if (admit) NGS_TRY(admit(admit_user, 0, plan_frame_fixed(bp) + plan_context(bp)));

  KeyBuf k1;
  k1.add(*g);
  k1.add(rp);
  k1.add(f->view_host.size());
  for (const ViewParams& vp : f->view_host) {  // everything but the pose, which the replay copies anew
    k1.add(vp.cam.W);
    k1.add(vp.cam.H);
    k1.add(vp.tile_base);
    k1.add(vp.pix_base);
  }
  for (const DevBuf* b : {&f->rec, &f->tile_count, &f->gkeys[0], &f->gkeys[1], &f->gvals[0], &f->gvals[1], &f->offsets,
                          &f->views, &ctx->hist, &ctx->scan_tmp, &ctx->total})
    k1.add(b->p);
  k1.add(f->h_views);
  k1.add(ctx->h_total);
  // asynchronous: no host synchronisation; phase 2 is sized by the frame's capacity (set by earlier renders)
  const bool async = f->async && f->pair_cap > 0 && !admit;
  NGS_TRY(run_phase(ctx, f, 0, k1, s, [&](cudaStream_t st) { return phase1(ctx, f, pl, st); }));
  cudaError_t e = cudaEventRecord(f->views_uploaded, s);
  uint32_t np = 0, cap = 0;
  const uint32_t* np_dev = nullptr;
  if (async) {
    if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("render: ") + cudaGetErrorString(e));
    cap = f->pair_cap;
    np_dev = reinterpret_cast<const uint32_t*>(ctx->total.p);  // low word of the pair count (< 2^31)
  } else {
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("reading the pair count: ") + cudaGetErrorString(e));
    const volatile uint64_t* mirror = ctx->h_total + kMirrorTotal;  // written by publish_words
    if (mirror[1] != 0) {  // a bounds check fired in an earlier call on this context
      const cudaError_t ze = cudaMemsetAsync(ctx->total.as<uint64_t>() + 1, 0, sizeof(uint64_t), s);
      if (ze != cudaSuccess)
        return fail(ctx, NGS_ERR_CUDA, std::string("clearing the device error word: ") + cudaGetErrorString(ze));
      return fail(ctx, NGS_ERR_DEVICE_CHECK, "a kernel bounds check fired in an earlier call on this context; its "
                                             "output was not valid");
    }
    const uint64_t P = mirror[0];
    if (P >= (1ull << 31)) return fail(ctx, NGS_ERR_INVALID_ARG, "more than 2^31 (tile, Gaussian) pairs");
    np = (uint32_t)P;
    if (admit)
      NGS_TRY(admit(admit_user, 1, plan_frame_pairs(plan_buffers(R, pl.n, (uint32_t)n_views, pl.ntiles, pix_total,
                                                                 rp.schedule, np))));
    // the capacity that graph replays and asynchronous renders reuse while the count fits
    if (np > f->pair_cap) f->pair_cap = (uint32_t)std::min<uint64_t>((uint64_t)np + np / 4 + 1024, (1ull << 31) - 1);
    // phase 2: exact sizes, or, for graph replays, the capacity
    cap = np;
    if (ctx->graphs) {
      cap = f->pair_cap;
      np_dev = reinterpret_cast<const uint32_t*>(ctx->total.p);
    }
  }
  const BufferPlan bp2 = plan_buffers(R, pl.n, (uint32_t)n_views, pl.ntiles, pix_total, rp.schedule, cap);
  for (int k = 0; k < 2; ++k) {
    NGS_TRY(ensure(ctx, f->ptile[k], bp2.pair_tile));
    NGS_TRY(ensure(ctx, f->pvals[k], bp2.pair_val));
  }
  NGS_TRY(ensure(ctx, ctx->hist, bp2.hist2));
  KeyBuf k2;
  k2.add(rp);
  k2.add(cap);
  k2.add(np_dev);
  k2.add(async);
  k2.add(f->g_final);
  k2.add(n_views == 1 ? pl.image : nullptr);  // a batch reads its outputs from the view table
  k2.add(n_views == 1 ? pl.overdraw : nullptr);
  k2.add(ctx->num_sms);
  for (const ViewParams& vp : f->view_host) {  // the tile sort's bit count follows the largest view
    k2.add(vp.tiles_x);
    k2.add(vp.tiles_y);
  }
  for (const DevBuf* b : {&f->rec, &f->gvals[0], &f->gvals[1], &f->offsets, &f->views, &f->ptile[0], &f->ptile[1],
                          &f->pvals[0], &f->pvals[1], &ctx->hist, &f->ranges, &f->work, &f->sched, &f->state})
    k2.add(b->p);
  if (async) k2.add(f->d_status);
  NGS_TRY(run_phase(ctx, f, 1, k2, s, [&](cudaStream_t st) { return phase2(ctx, f, pl, cap, np_dev, async, st); }));
  if (async) {
    e = cudaEventRecord(f->done, s);
    if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("render: ") + cudaGetErrorString(e));
    f->pending = true;
  }
  f->last_async = async;

  f->n = pl.n;
  if (!async) f->pairs = np;  // an asynchronous render's count is known once ngs_frame_status has read it
  f->n_views = n_views;
  f->n_pixels = (int64_t)pix_total;
  f->rp = rp;
  f->has_render = true;
  return NGS_OK;
}

extern "C" {

NGS_API void ngs_default_options(ngs_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->alpha_min = 1.0f / 255.0f;
  o->alpha_max = 0.99f;
  o->t_eps = 1e-4f;
  o->dilation = 0.3f;
  o->near_plane = 0.2f;
  o->tile_w = 16;
  o->tile_h = 16;
  o->max_splats = 0;
}

NGS_API int ngs_create(ngs_ctx** out) {
  if (!out) return NGS_ERR_INVALID_ARG;
  *out = nullptr;
  ngs_ctx* ctx = new (std::nothrow) ngs_ctx();
  if (!ctx) return NGS_ERR_OUT_OF_MEMORY;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&ctx->h_total, kMirrorWords * sizeof(uint64_t), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&ctx->d_h_total, ctx->h_total, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (ctx->h_total) cudaFreeHost(ctx->h_total);
    delete ctx;
    return NGS_ERR_CUDA;
  }
  *out = ctx;
  return NGS_OK;
}

NGS_API void ngs_destroy(ngs_ctx* ctx) {
  if (!ctx) return;
  cudaDeviceSynchronize();
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  free_buf(ctx->hist);
  free_buf(ctx->scan_tmp);
  free_buf(ctx->grad2d);
  free_buf(ctx->total);
  free_buf(ctx->flush);
  free_buf(ctx->loss_tmp);
  free_buf(ctx->densify_tmp);
  free_buf(ctx->densify_totals);
  free_buf(ctx->check_word);
  if (ctx->h_total) cudaFreeHost(ctx->h_total);
  for (auto& p : ctx->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : ctx->event_pool) cudaEventDestroy(e);
  delete ctx;
}

NGS_API const char* ngs_last_error(const ngs_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

NGS_API int ngs_frame_create(ngs_ctx* ctx, ngs_frame** out) {
  if (!ctx || !out) return NGS_ERR_INVALID_ARG;
  ngs_frame* f = new (std::nothrow) ngs_frame();
  if (!f) return fail(ctx, NGS_ERR_OUT_OF_MEMORY, "host allocation of a frame failed");
  f->ctx = ctx;
  *out = f;
  return NGS_OK;
}

NGS_API void ngs_frame_destroy(ngs_frame* f) {
  if (!f) return;
  cudaDeviceSynchronize();
  DevBuf* bufs[] = {&f->rec,     &f->tile_count, &f->gkeys[0], &f->gkeys[1], &f->gvals[0], &f->gvals[1],
                    &f->offsets, &f->ptile[0],   &f->ptile[1], &f->pvals[0], &f->pvals[1], &f->ranges,
                    &f->state,   &f->views,      &f->keys64,   &f->work,     &f->sched};
  for (DevBuf* b : bufs) free_buf(*b);
  if (f->h_views) cudaFreeHost(f->h_views);
  if (f->views_uploaded) cudaEventDestroy(f->views_uploaded);
  if (f->h_status) cudaFreeHost(f->h_status);
  if (f->done) cudaEventDestroy(f->done);
  for (GraphSlot& g : f->graph)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  delete f;
}

NGS_API int ngs_frame_set_async(ngs_frame* f, int enable) {
  if (!f) return NGS_ERR_INVALID_ARG;
  if (enable && !f->h_status) {
    void* dev_alias = nullptr;
    cudaError_t e = cudaHostAlloc((void**)&f->h_status, 3 * sizeof(uint64_t), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&dev_alias, f->h_status, 0);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (f->h_status) cudaFreeHost(f->h_status);
      f->h_status = nullptr;
      f->done = nullptr;
      return fail(f->ctx, NGS_ERR_CUDA, std::string("asynchronous frame: ") + cudaGetErrorString(e));
    }
    memset(f->h_status, 0, 3 * sizeof(uint64_t));
    f->d_status = static_cast<uint64_t*>(dev_alias);
  }
  f->async = enable != 0;
  return NGS_OK;
}

NGS_API int ngs_frame_status(ngs_frame* f, int64_t* pairs) {
  if (!f) return NGS_ERR_INVALID_ARG;
  if (!f->has_render) return fail(f->ctx, NGS_ERR_INVALID_ARG, "frame holds no render");
  int rc = NGS_OK;
  if (f->pending) {
    cudaError_t e = cudaEventSynchronize(f->done);
    if (e != cudaSuccess) return fail(f->ctx, NGS_ERR_CUDA, std::string("frame status: ") + cudaGetErrorString(e));
    volatile uint64_t* st = f->h_status;  // written by finish_async_kernel
    const uint64_t most = st[0], err = st[1], last = st[2];
    st[0] = 0;
    st[1] = 0;
    f->pending = false;
    if (f->last_async) f->pairs = (int64_t)last;
    if (err & kCheckCapacity) {
      f->pair_cap = (uint32_t)std::min<uint64_t>(most + most / 4 + 1024, (1ull << 31) - 1);
      rc = fail(f->ctx, NGS_ERR_CAPACITY, "an asynchronous render met " + std::to_string(most) +
                                              " pairs, more than its frame's capacity; the capacity has grown");
    } else if (err) {
      rc = fail(f->ctx, NGS_ERR_DEVICE_CHECK, "a kernel bounds check fired in an asynchronous render; its output "
                                              "was not valid");
    }
  }
  if (pairs) *pairs = f->pairs;
  return rc;
}

NGS_API int ngs_render(ngs_ctx* ctx, ngs_frame* f, const ngs_gaussians* g, const ngs_camera* cam,
                       const ngs_model* model, const ngs_options* o, float* image, int32_t* overdraw, void* stream) {
  if (!ctx) return NGS_ERR_INVALID_ARG;
  return render_views(ctx, f, g, cam, 1, model, o, image, overdraw, (cudaStream_t)stream);
}

NGS_API int ngs_render_batch(ngs_ctx* ctx, ngs_frame* f, const ngs_gaussians* g, const ngs_camera* cams,
                             int32_t n_views, const ngs_model* model, const ngs_options* o, float* images,
                             int32_t* overdraw, void* stream) {
  if (!ctx) return NGS_ERR_INVALID_ARG;
  return render_views(ctx, f, g, cams, n_views, model, o, images, overdraw, (cudaStream_t)stream);
}

NGS_API int ngs_render_backward(ngs_ctx* ctx, const ngs_frame* f, const ngs_gaussians* g, const float* dl_dimage,
                                const ngs_grads* out, void* stream) {
  return ngs::backward_frame(ctx, f, g, dl_dimage, out, (cudaStream_t)stream);
}

}  // extern "C"

int ngs::backward_frame(ngs_ctx* ctx, const ngs_frame* f, const ngs_gaussians* g, const float* dl_dimage,
                        const ngs_grads* out, cudaStream_t s) {
  if (!ctx) return NGS_ERR_INVALID_ARG;
  if (!f || f->ctx != ctx || !f->has_render) return fail(ctx, NGS_ERR_INVALID_ARG, "frame holds no render");
  if (!g || !dl_dimage || !out) return fail(ctx, NGS_ERR_INVALID_ARG, "null argument");
  if (g->n != f->n || g->sh_degree != f->rp.sh_degree)
    return fail(ctx, NGS_ERR_INVALID_ARG, "Gaussians do not match the rendered frame");
  if (g->n > 0 && (!out->d_means || !out->d_log_scales || !out->d_quats || !out->d_opacity_logits || !out->d_sh))
    return fail(ctx, NGS_ERR_INVALID_ARG, "null gradient array");
  const uint32_t R = f->rp.n_records;
  NGS_TRY(ensure(ctx, ctx->grad2d, plan_buffers(R, 0, 1, 0, 0, 0, 0).grad2d));
  // the replay adds into the record gradients: a failed clear must not let it add onto stale values
  cudaError_t e = cudaMemsetAsync(ctx->grad2d.p, 0, sizeof(float4) * 3 * (size_t)R, s);
  if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("clearing the record gradients: ") + cudaGetErrorString(e));
  const ViewParams* views = f->views.as<ViewParams>();
  const uint32_t* work = nullptr;
  uint32_t* counter = nullptr;
  if (f->rp.schedule == NGS_SCHEDULE_PERSISTENT) {
    work = f->work.as<uint32_t>();
    counter = f->sched.as<uint32_t>() + 1;
    e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("clearing the work counter: ") + cudaGetErrorString(e));
  }
  cudaEvent_t ev;
  stage_begin(ctx, s, 6, &ev);
  launch_composite_backward(f->rec.as<float4>(), f->pvals[f->p_final].as<uint32_t>(), f->ranges.as<uint2>(), f->rp,
                            views, dl_dimage, f->state.as<float4>(), ctx->grad2d.as<float4>(), work, counter,
                            ctx->num_sms, s);
  stage_end(ctx, s, 6, ev, 1);
  NGS_TRY(check_launch(ctx, "composite backward"));
  stage_begin(ctx, s, 7, &ev);
  launch_project_backward(*g, views, f->view_host[0].cam, f->rp, f->tile_count.as<uint32_t>(), ctx->grad2d.as<float4>(), *out,
                          ctx->num_sms, s);
  stage_end(ctx, s, 7, ev, g->n ? 1 : 0);
  NGS_TRY(check_launch(ctx, "projection backward"));
  return NGS_OK;
}

extern "C" {

NGS_API int ngs_frame_view_get(const ngs_frame* fc, ngs_frame_view* out) {
  if (!fc || !out) return NGS_ERR_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  if (!fc->has_render) return NGS_ERR_INVALID_ARG;
  // the hot path sorts 32-bit tile indices; the 64-bit keys are composed here, after the device is idle
  ngs_frame* f = const_cast<ngs_frame*>(fc);
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(f->ctx, NGS_ERR_CUDA, "frame view: device error");
  if (f->pending && f->last_async) {  // an asynchronous render's count (its status stays unread)
    const uint64_t last = static_cast<volatile uint64_t*>(f->h_status)[2];
    f->pairs = (int64_t)std::min<uint64_t>(last, f->pair_cap);
  }
  uint32_t np = (uint32_t)f->pairs;
  if (ensure(f->ctx, f->keys64, sizeof(uint64_t) * (size_t)std::max(np, 1u)) != NGS_OK) return NGS_ERR_OUT_OF_MEMORY;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) {
    launch_compose_keys(f->ptile[f->p_final].as<uint32_t>(), f->pvals[f->p_final].as<uint32_t>(), f->rec.as<float4>(),
                        f->views.as<ViewParams>(), (uint32_t)f->n, (uint32_t)f->n_views, np, f->keys64.as<uint64_t>(),
                        nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
  if (e != cudaSuccess) return fail(f->ctx, NGS_ERR_CUDA, std::string("composing keys: ") + cudaGetErrorString(e));
  out->n_gaussians = f->n;
  out->n_pairs = f->pairs;
  out->tiles_x = f->view_host[0].tiles_x;
  out->tiles_y = f->view_host[0].tiles_y;
  out->width = f->view_host[0].cam.W;
  out->height = f->view_host[0].cam.H;
  out->n_views = f->n_views;
  out->view_pixel_base = f->pix_base.data();
  out->view_tile_base = f->tile_base.data();
  out->log2_alpha_min = f->rp.log2_alpha_min;
  out->records = f->rec.as<float>();
  out->keys = f->keys64.as<uint64_t>();
  out->values = f->pvals[f->p_final].as<uint32_t>();
  out->ranges = f->ranges.as<uint32_t>();
  out->pixel_state = f->state.as<float>();
  return NGS_OK;
}

NGS_API int ngs_set_graphs(ngs_ctx* ctx, int enable) {
  if (!ctx) return NGS_ERR_INVALID_ARG;
  ctx->graphs = enable != 0;
  return NGS_OK;
}

NGS_API int64_t ngs_graph_captures(const ngs_ctx* ctx) { return ctx ? ctx->graph_captures : 0; }

NGS_API int ngs_set_timing(ngs_ctx* ctx, int enable) {
  if (!ctx) return NGS_ERR_INVALID_ARG;
  ctx->timing = enable != 0;
  return NGS_OK;
}

NGS_API int ngs_stage_times(ngs_ctx* ctx, double* ms, int64_t* launches, int32_t n) {
  if (!ctx) return NGS_ERR_INVALID_ARG;
  for (auto& p : ctx->pending) {
    float t = 0.f;
    cudaEventSynchronize(p.b);
    if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) ctx->stage_ms[p.stage] += t;
    ctx->event_pool.push_back(p.a);
    ctx->event_pool.push_back(p.b);
  }
  ctx->pending.clear();
  for (int i = 0; i < n && i < NGS_NUM_STAGES; ++i) {
    if (ms) ms[i] = ctx->stage_ms[i];
    if (launches) launches[i] = ctx->stage_launches[i];
  }
  return NGS_NUM_STAGES;
}

NGS_API void ngs_reset_stage_times(ngs_ctx* ctx) {
  if (!ctx) return;
  ngs_stage_times(ctx, nullptr, nullptr, 0);
  for (int i = 0; i < NGS_NUM_STAGES; ++i) {
    ctx->stage_ms[i] = 0;
    ctx->stage_launches[i] = 0;
  }
}

NGS_API int64_t ngs_launch_count(const ngs_ctx* ctx) { return ctx ? ctx->launches : 0; }

NGS_API int ngs_set_checked(ngs_ctx* ctx, int enable) {
  if (!ctx) return NGS_ERR_INVALID_ARG;
  ctx->checked = enable != 0;
  return NGS_OK;
}

NGS_API int ngs_workspace_bytes(int64_t n, const ngs_camera* cams, int32_t n_views, const ngs_options* o,
                                int64_t n_pairs, ngs_workspace* out) {
  if (!cams || !o || !out || n < 0 || n >= (1ll << 31) || n_pairs < 0 || n_pairs >= (1ll << 31))
    return NGS_ERR_INVALID_ARG;
  if (n_views < 1 || n_views > kMaxViews) return NGS_ERR_INVALID_ARG;
  const bool tile_ok = (o->tile_w == 8 && o->tile_h == 8) || (o->tile_w == 16 && o->tile_h == 16) ||
                       (o->tile_w == 16 && o->tile_h == 32);
  if (!tile_ok) return NGS_ERR_INVALID_ARG;
  uint64_t tiles = 0, pix = 0;
  for (int v = 0; v < n_views; ++v) {
    if (check_camera(nullptr, &cams[v]) != NGS_OK) return NGS_ERR_INVALID_ARG;
    tiles += (uint64_t)((cams[v].width + o->tile_w - 1) / o->tile_w) * ((cams[v].height + o->tile_h - 1) / o->tile_h);
    pix += (uint64_t)cams[v].width * cams[v].height;
  }
  const uint64_t R = (uint64_t)n * (uint64_t)n_views;
  if (R >= (1ull << 32)) return NGS_ERR_INVALID_ARG;
  const BufferPlan b = plan_buffers(R, (uint32_t)n, (uint32_t)n_views, tiles, pix, o->schedule, (uint64_t)n_pairs);
  out->frame_fixed = plan_frame_fixed(b);
  out->frame_pairs = plan_frame_pairs(b);
  out->context = plan_context(b);
  out->backward = fresh_bytes(b.grad2d);
  out->total = out->frame_fixed + out->frame_pairs + out->context + out->backward;
  return NGS_OK;
}

NGS_API int ngs_memory_usage(const ngs_ctx* ctx, const ngs_frame* f, size_t* ctx_bytes, size_t* frame_bytes) {
  if (ctx_bytes) {
    *ctx_bytes = 0;
    if (ctx)
      for (const DevBuf* b : {&ctx->hist, &ctx->scan_tmp, &ctx->grad2d, &ctx->total, &ctx->flush, &ctx->loss_tmp,
                              &ctx->densify_tmp, &ctx->densify_totals, &ctx->check_word})
        *ctx_bytes += b->p ? b->cap : 0;
  }
  if (frame_bytes) {
    *frame_bytes = 0;
    if (f)
      for (const DevBuf* b : {&f->rec, &f->tile_count, &f->gkeys[0], &f->gkeys[1], &f->gvals[0], &f->gvals[1],
                              &f->offsets, &f->ptile[0], &f->ptile[1], &f->pvals[0], &f->pvals[1], &f->ranges,
                              &f->state, &f->views, &f->keys64, &f->work, &f->sched})
        *frame_bytes += b->p ? b->cap : 0;
  }
  return NGS_OK;
}

}  // extern "C"
