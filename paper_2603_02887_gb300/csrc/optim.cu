// Training-step kernels (Sec. 5.1 "Optimization" and "Densification"): Adam over every parameter array in
// one launch, the accumulation of each Gaussian's positional-gradient magnitude, and split / prune
// compaction into new arrays.
//
// Adam (Kingma and Ba): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, step = lr m^ / (sqrt(v^) + eps) with
// the bias-corrected m^ = m / (1 - b1^t), v^ = v / (1 - b2^t); "bounded": the step is clipped to [-lr, lr].
//
// Densification: Gaussian i is pruned when sigmoid(logit) < min_opacity or max_k exp(s_k) < min_scale; else
// split when its mean positional-gradient magnitude accum / count exceeds the threshold (count > 0); else
// kept. Splits are granted in index order while the total stays within max_gaussians. A split replaces the
// Gaussian by two children at mu +- (sigma_a / 2) r_a along its longest axis a (r_a the rotation's column,
// sigma_a = exp(s_a)), with sigma_a scaled by sqrt(3)/2 so that the pair keeps the parent's variance along
// r_a (sigma_a'^2 + (sigma_a / 2)^2 = sigma_a^2); the other scales, the rotation, the opacity and the SH are
// the parent's. Kept Gaussians keep their Adam moments; children start from zero.
#include <math.h>

#include <algorithm>

#include "ngs_internal.cuh"

namespace ngs {
namespace {

struct ParamPtrs {
  float* p[5];
};

// element e of the virtual concatenation means | log_scales | quats | opacity_logits | sh
__device__ __forceinline__ int group_of(int64_t e, const int64_t (&end)[5], int64_t& local) {
  int gi = 0;
  while (gi < 4 && e >= end[gi]) ++gi;
  local = e - (gi ? end[gi - 1] : 0);
  return gi;
}

struct AdamArgs {
  ParamPtrs param, grad, m, v;
  int64_t end[5];
  float lr[5];
  float b1, b2, eps, c1, c2;  // c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t)
  int bounded;
};

__global__ void adam_kernel(AdamArgs a, int64_t total) {
  pdl_wait();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i;
    const int gi = group_of(e, a.end, i);
    const float g = a.grad.p[gi][i];
    const float m = fmaf(a.b1, a.m.p[gi][i], (1.f - a.b1) * g);
    const float v = fmaf(a.b2, a.v.p[gi][i], (1.f - a.b2) * g * g);
    a.m.p[gi][i] = m;
    a.v.p[gi][i] = v;
    float step = a.lr[gi] * (m * a.c1) / (sqrtf(v * a.c2) + a.eps);
    if (a.bounded) step = fminf(fmaxf(step, -a.lr[gi]), a.lr[gi]);
    a.param.p[gi][i] -= step;
  }
}

__global__ void accumulate_kernel(const float* __restrict__ d_means, int64_t n, float* __restrict__ accum,
                                  float* __restrict__ count) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float x = d_means[3 * i], y = d_means[3 * i + 1], z = d_means[3 * i + 2];
    const float norm = sqrtf(x * x + y * y + z * z);
    if (norm > 0.f) {
      accum[i] += norm;
      count[i] += 1.f;
    }
  }
}

// decision per Gaussian: 0 prune, 1 keep, 2 split candidate
__global__ void densify_decide_kernel(const float* __restrict__ logits, const float* __restrict__ log_scales,
                                      const float* __restrict__ accum, const float* __restrict__ count, int64_t n,
                                      ngs_densify_cfg cfg, uint32_t* __restrict__ decision,
                                      uint32_t* __restrict__ is_split) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float op = 1.f / (1.f + expf(-logits[i]));
  const float smax = expf(fmaxf(log_scales[3 * i], fmaxf(log_scales[3 * i + 1], log_scales[3 * i + 2])));
  uint32_t d = 1;
  if (cfg.prune && (op < cfg.min_opacity || smax < cfg.min_scale)) d = 0;
  else if (cfg.split && count[i] > 0.f && accum[i] / count[i] > cfg.grad_threshold) d = 2;
  decision[i] = d;
  is_split[i] = d == 2 ? 1u : 0u;
}

__device__ __forceinline__ void quat_axis(const float* q, int a, float* r) {
  const float n = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const float w = q[0] * n, x = q[1] * n, y = q[2] * n, z = q[3] * n;
  // column a of the rotation matrix of the unit quaternion (w, x, y, z)
  if (a == 0) {
    r[0] = 1.f - 2.f * (y * y + z * z);
    r[1] = 2.f * (x * y + w * z);
    r[2] = 2.f * (x * z - w * y);
  } else if (a == 1) {
    r[0] = 2.f * (x * y - w * z);
    r[1] = 1.f - 2.f * (x * x + z * z);
    r[2] = 2.f * (y * z + w * x);
  } else {
    r[0] = 2.f * (x * z + w * y);
    r[1] = 2.f * (y * z - w * x);
    r[2] = 1.f - 2.f * (x * x + y * y);
  }
}

struct DensifyArgs {
  ParamPtrs src, src_m, src_v, dst, dst_m, dst_v;
  int K3;  // 3 (sh_degree + 1)^2
};

__global__ void iota_kernel(uint32_t* __restrict__ out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (uint32_t)i;
}

// splits allowed under the cap: min(candidates, max(0, cap - survivors)); survivors = n - pruned
__global__ void densify_allowed_kernel(const uint64_t* __restrict__ cand_total,
                                       const uint64_t* __restrict__ prune_total, int64_t n, int64_t cap,
                                       uint32_t* __restrict__ allowed) {
  const int64_t survivors = n - (int64_t)*prune_total;
  const int64_t room = cap > survivors ? cap - survivors : 0;
  *allowed = (uint32_t)min((int64_t)*cand_total, room);
}

// number of pruned Gaussians (decision 0), one atomic per warp
__global__ void count_pruned_kernel(const uint32_t* __restrict__ decision, int64_t n, uint64_t* __restrict__ pruned) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const uint32_t b = __ballot_sync(0xFFFFFFFFu, i < n && decision[i] == 0);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(reinterpret_cast<unsigned long long*>(pruned), (unsigned long long)__popc(b));
}

// output count per Gaussian: 0 pruned, 2 a granted split, else 1
__global__ void densify_count_kernel(const uint32_t* __restrict__ decision, const uint32_t* __restrict__ rank,
                                     const uint32_t* __restrict__ allowed, int64_t n, uint32_t* __restrict__ outc) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t d = decision[i];
  outc[i] = d == 0 ? 0u : (d == 2 && rank[i] < *allowed ? 2u : 1u);
}

__global__ void densify_apply_kernel(DensifyArgs a, const uint32_t* __restrict__ outc, const uint32_t* __restrict__ pos,
                                     int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t c = outc[i];
  if (c == 0) return;
  const int64_t o = pos[i];
  static const int kWidth[4] = {3, 3, 4, 1};  // means, log_scales, quats, opacity_logits
  if (c == 1) {
    for (int gi = 0; gi < 5; ++gi) {
      const int w = gi < 4 ? kWidth[gi] : a.K3;
      for (int k = 0; k < w; ++k) {
        a.dst.p[gi][o * w + k] = a.src.p[gi][i * w + k];
        a.dst_m.p[gi][o * w + k] = a.src_m.p[gi][i * w + k];
        a.dst_v.p[gi][o * w + k] = a.src_v.p[gi][i * w + k];
      }
    }
    return;
  }
  // split along the longest axis
  const float* ls = a.src.p[1] + 3 * i;
  const int ax = ls[0] >= ls[1] ? (ls[0] >= ls[2] ? 0 : 2) : (ls[1] >= ls[2] ? 1 : 2);
  float r[3];
  quat_axis(a.src.p[2] + 4 * i, ax, r);
  const float half = 0.5f * expf(ls[ax]);
  for (int child = 0; child < 2; ++child) {
    const int64_t oc = o + child;
    const float sgn = child == 0 ? 1.f : -1.f;
    for (int gi = 0; gi < 5; ++gi) {
      const int w = gi < 4 ? kWidth[gi] : a.K3;
      for (int k = 0; k < w; ++k) {
        float val = a.src.p[gi][i * w + k];
        if (gi == 0) val += sgn * half * r[k];
        if (gi == 1 && k == ax) val += logf(0.8660254037844386f);  // sigma_a sqrt(3)/2
        a.dst.p[gi][oc * w + k] = val;
        a.dst_m.p[gi][oc * w + k] = 0.f;
        a.dst_v.p[gi][oc * w + k] = 0.f;
      }
    }
  }
}

ParamPtrs ptrs(const ngs_grads& g) { return ParamPtrs{{g.d_means, g.d_log_scales, g.d_quats, g.d_opacity_logits, g.d_sh}}; }

bool complete(const ngs_grads* g) {
  return g && g->d_means && g->d_log_scales && g->d_quats && g->d_opacity_logits && g->d_sh;
}

unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1 << 20)); }

}  // namespace
}  // namespace ngs

using namespace ngs;

extern "C" {

NGS_API int ngs_adam_step(ngs_ctx* ctx, int64_t n, int32_t sh_degree, const ngs_grads* params, const ngs_grads* grads,
                          const ngs_grads* m, const ngs_grads* v, const ngs_adam* cfg, void* stream) {
  if (!ctx) return NGS_ERR_INVALID_ARG;
  if (n < 0 || sh_degree < 0 || sh_degree > 3 || !cfg || cfg->step < 1 || !(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) ||
      !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) || !(cfg->eps > 0.f))
    return fail(ctx, NGS_ERR_INVALID_ARG, "adam: n, sh_degree or the configuration out of range");
  if (n == 0) return NGS_OK;
  if (!complete(params) || !complete(grads) || !complete(m) || !complete(v))
    return fail(ctx, NGS_ERR_INVALID_ARG, "adam: null array");
  const int K3 = 3 * (sh_degree + 1) * (sh_degree + 1);
  AdamArgs a;
  a.param = ptrs(*params);
  a.grad = ptrs(*grads);
  a.m = ptrs(*m);
  a.v = ptrs(*v);
  const int64_t width[5] = {3, 3, 4, 1, K3};
  int64_t acc = 0;
  for (int gi = 0; gi < 5; ++gi) {
    acc += width[gi] * n;
    a.end[gi] = acc;
    a.lr[gi] = cfg->lr[gi];
  }
  a.b1 = cfg->beta1;
  a.b2 = cfg->beta2;
  a.eps = cfg->eps;
  a.c1 = (float)(1.0 / (1.0 - pow((double)cfg->beta1, (double)cfg->step)));
  a.c2 = (float)(1.0 / (1.0 - pow((double)cfg->beta2, (double)cfg->step)));
  a.bounded = cfg->bounded != 0;
  launch_pdl(adam_kernel, grid_for(acc), 256, 0, (cudaStream_t)stream, a, acc);
  ctx->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("adam launch: ") + cudaGetErrorString(e));
  return NGS_OK;
}

NGS_API int ngs_accumulate_grad_norm(ngs_ctx* ctx, int64_t n, const float* d_means, float* accum, float* count,
                                     void* stream) {
  if (!ctx) return NGS_ERR_INVALID_ARG;
  if (n < 0 || (n > 0 && (!d_means || !accum || !count)))
    return fail(ctx, NGS_ERR_INVALID_ARG, "accumulate: null array or n < 0");
  if (n == 0) return NGS_OK;
  launch_pdl(accumulate_kernel, grid_for(n), 256, 0, (cudaStream_t)stream, d_means, n, accum, count);
  ctx->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("accumulate launch: ") + cudaGetErrorString(e));
  return NGS_OK;
}

NGS_API int ngs_densify(ngs_ctx* ctx, int64_t n, int32_t sh_degree, const ngs_grads* params, const ngs_grads* m,
                        const ngs_grads* v, const float* accum, const float* count, const ngs_densify_cfg* cfg,
                        int64_t capacity, const ngs_grads* out_params, const ngs_grads* out_m, const ngs_grads* out_v,
                        int64_t* n_out, void* stream) {
  if (!ctx) return NGS_ERR_INVALID_ARG;
  if (!cfg || !n_out || n < 0 || n >= (1ll << 30) || sh_degree < 0 || sh_degree > 3 || cfg->max_gaussians < 0)
    return fail(ctx, NGS_ERR_INVALID_ARG, "densify: null argument or n, sh_degree, max_gaussians out of range");
  const int64_t needed = std::min<int64_t>(2 * n, std::max<int64_t>(n, cfg->max_gaussians));
  if (capacity < needed)
    return fail(ctx, NGS_ERR_INVALID_ARG, "densify: output capacity below min(2 n, max(n, max_gaussians))");
  *n_out = 0;
  if (n == 0) return NGS_OK;
  if (!complete(params) || !complete(m) || !complete(v) || !complete(out_params) || !complete(out_m) ||
      !complete(out_v) || !accum || !count)
    return fail(ctx, NGS_ERR_INVALID_ARG, "densify: null array");
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t un = (uint32_t)n;
  // scratch: decision, candidate flags, their scan, output counts, their scan, identity order (u32 each),
  // allowed count; the scan's block sums and totals in the context's scan scratch
  const size_t words = 6 * ((size_t)un + 1) + 4;
  int rc = ensure(ctx, ctx->densify_tmp, sizeof(uint32_t) * words);
  if (rc == NGS_OK) rc = ensure(ctx, ctx->scan_tmp, sizeof(uint64_t) * scan_tmp_words(un));
  if (rc == NGS_OK) rc = ensure(ctx, ctx->densify_totals, 3 * sizeof(uint64_t));
  if (rc != NGS_OK) return rc;
  uint32_t* decision = ctx->densify_tmp.as<uint32_t>();
  uint32_t* cand = decision + (un + 1);
  uint32_t* rank = cand + (un + 1);
  uint32_t* outc = rank + (un + 1);
  uint32_t* pos = outc + (un + 1);
  uint32_t* iota = pos + (un + 1);
  uint32_t* allowed = iota + (un + 1);
  uint64_t* totals = ctx->densify_totals.as<uint64_t>();
  const unsigned blocks = (un + 255) / 256;
  int launches = 0;
  iota_kernel<<<blocks, 256, 0, s>>>(iota, n);
  densify_decide_kernel<<<blocks, 256, 0, s>>>(params->d_opacity_logits, params->d_log_scales, accum, count, n, *cfg,
                                               decision, cand);
  launches += 2;
  cudaError_t me = launch_scan_counts(cand, iota, un, rank, ctx->scan_tmp.as<uint64_t>(), &totals[0], s, &launches);
  if (me == cudaSuccess) me = cudaMemsetAsync(&totals[1], 0, sizeof(uint64_t), s);
  if (me != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("densify: ") + cudaGetErrorString(me));
  count_pruned_kernel<<<blocks, 256, 0, s>>>(decision, n, &totals[1]);
  densify_allowed_kernel<<<1, 1, 0, s>>>(&totals[0], &totals[1], n, cfg->max_gaussians, allowed);
  densify_count_kernel<<<blocks, 256, 0, s>>>(decision, rank, allowed, n, outc);
  launches += 3;
  me = launch_scan_counts(outc, iota, un, pos, ctx->scan_tmp.as<uint64_t>(), &totals[2], s, &launches);
  if (me != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("densify: ") + cudaGetErrorString(me));
  DensifyArgs da;
  da.src = ptrs(*params);
  da.src_m = ptrs(*m);
  da.src_v = ptrs(*v);
  da.dst = ptrs(*out_params);
  da.dst_m = ptrs(*out_m);
  da.dst_v = ptrs(*out_v);
  da.K3 = 3 * (sh_degree + 1) * (sh_degree + 1);
  densify_apply_kernel<<<blocks, 256, 0, s>>>(da, outc, pos, n);
  launches += 1;
  ctx->launches += launches;
  publish_words(ctx, &totals[2], 1, kMirrorDensify, s);  // the new count, through the mapped mirror
  ctx->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("densify: ") + cudaGetErrorString(e));
  *n_out = (int64_t)static_cast<volatile uint64_t*>(ctx->h_total)[kMirrorDensify];
  return NGS_OK;
}

}  // extern "C"
