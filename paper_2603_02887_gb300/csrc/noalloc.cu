// ngs_render_backward_static: the path-replay backward without any device allocation.
//
// ngs_render_backward keeps its per-Gaussian splat-record gradients (3 float4 per Gaussian) in scratch
// that the context allocates with cudaMalloc on first use and grows on demand. Some callers cannot let
// a library allocate: applications that own a fixed device-memory budget (a server that reserves its
// pool up front, a host program that forbids third-party allocations), and latency-critical loops in
// which cudaMalloc / cudaFree would synchronise the device and stall other streams. This variant keeps
// that scratch in a fixed static device array instead, and allocates nothing.
//
// Limits and behaviour:
//  * at most kStaticMaxRecords = 262,144 splat records (Gaussians x views) per call (the array is 12 MiB);
//    larger frames are rejected with NGS_ERR_INVALID_ARG and a message that names the limit;
//  * every GPU that loads this library holds the array until the process exits;
//  * all calls on a device share the one array and it keeps the previous call's contents, so each call
//    clears the part it uses (cudaMemsetAsync) before use, and calls whose work overlaps on the GPU
//    (different streams or host threads without ordering between them) race on it;
//  * the first call on a device, with that device current, looks up the array's device address with
//    cudaGetSymbolAddress (host code cannot use the symbol itself as a device pointer); make that first
//    call before any stream capture;
//  * the context's device must be the current device (else NGS_ERR_INVALID_ARG): the array is looked up on
//    the current device, and the frame's buffers live on the context's.
#include <mutex>

#include "ngs_internal.cuh"

namespace {

constexpr int64_t kStaticMaxRecords = 262144;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float4 g_static_grad2d[3 * kStaticMaxRecords];

std::mutex g_mutex;
void* g_device_ptr[kMaxDevices] = {};

// Device address of g_static_grad2d on the context's device, which must be current (looked up once per device).
int static_scratch(ngs_ctx* ctx, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ngs::fail(ctx, NGS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != ctx->device)
    return ngs::fail(ctx, NGS_ERR_INVALID_ARG, "ngs_render_backward_static: the context's device (" +
                                                   std::to_string(ctx->device) + ") is not the current device (" +
                                                   std::to_string(dev) + ")");
  if (dev < 0 || dev >= kMaxDevices) return ngs::fail(ctx, NGS_ERR_INVALID_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_device_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_grad2d);
    if (e != cudaSuccess || !p)
      return ngs::fail(ctx, NGS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_device_ptr[dev] = p;
  }
  *out = g_device_ptr[dev];
  return NGS_OK;
}

}  // namespace

extern "C" NGS_API int ngs_render_backward_static(ngs_ctx* ctx, const ngs_frame* f, const ngs_gaussians* g,
                                                  const float* dl_dimage, const ngs_grads* out, void* stream) {
  using namespace ngs;
  if (!ctx) return NGS_ERR_INVALID_ARG;
  if (!f || f->ctx != ctx || !f->has_render) return fail(ctx, NGS_ERR_INVALID_ARG, "frame holds no render");
  if (!g || !dl_dimage || !out) return fail(ctx, NGS_ERR_INVALID_ARG, "null argument");
  if (g->n != f->n || g->sh_degree != f->rp.sh_degree)
    return fail(ctx, NGS_ERR_INVALID_ARG, "Gaussians do not match the rendered frame");
  if ((int64_t)f->rp.n_records > kStaticMaxRecords)
    return fail(ctx, NGS_ERR_INVALID_ARG,
                "ngs_render_backward_static handles at most 262144 splat records (Gaussians x views; static "
                "scratch of 12 MiB); use ngs_render_backward for larger scenes");
  if (g->n > 0 && (!out->d_means || !out->d_log_scales || !out->d_quats || !out->d_opacity_logits || !out->d_sh))
    return fail(ctx, NGS_ERR_INVALID_ARG, "null gradient array");
  void* scratch = nullptr;
  int rc = static_scratch(ctx, &scratch);
  if (rc != NGS_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  size_t n = (size_t)f->n;
  float4* grad2d = reinterpret_cast<float4*>(scratch);
  cudaError_t e = cudaMemsetAsync(grad2d, 0, sizeof(float4) * 3 * (size_t)f->rp.n_records, s);
  if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("clearing the scratch: ") + cudaGetErrorString(e));
  const ViewParams* views = f->views.as<ViewParams>();
  const uint32_t* work = nullptr;
  uint32_t* counter = nullptr;
  if (f->rp.schedule == NGS_SCHEDULE_PERSISTENT) {  // the frame's own work list and counter (no allocation)
    work = f->work.as<uint32_t>();
    counter = f->sched.as<uint32_t>() + 1;
    e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("clearing the work counter: ") + cudaGetErrorString(e));
  }
  launch_composite_backward(f->rec.as<float4>(), f->pvals[f->p_final].as<uint32_t>(), f->ranges.as<uint2>(), f->rp,
                            views, dl_dimage, f->state.as<float4>(), grad2d, work, counter, ctx->num_sms, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("composite backward: ") + cudaGetErrorString(e));
  ctx->launches += 1;
  ctx->stage_launches[6] += 1;
  if (n) {
    launch_project_backward(*g, views, f->view_host[0].cam, f->rp, f->tile_count.as<uint32_t>(), grad2d, *out,
                            ctx->num_sms, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("projection backward: ") + cudaGetErrorString(e));
    ctx->launches += 1;
    ctx->stage_launches[7] += 1;
  }
  return NGS_OK;
}
