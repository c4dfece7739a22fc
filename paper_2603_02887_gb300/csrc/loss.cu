// Image loss of the training step (Sec. 5.1 "Loss"): L = (1 - lambda) L1 + lambda (1 - SSIM), with L1 the
// mean absolute difference and SSIM the mean structural similarity (Wang et al. 2004) over pixels and
// channels, with the 11 x 11 Gaussian window (sigma 1.5) and zero padding of 3D Gaussian splatting, and
// its gradient w.r.t. the rendered image.
//
// Per channel, with windowed moments mx = G * x, my = G * y, sxx = G * x^2, syy = G * y^2, sxy = G * xy:
//   s = (2 mx my + C1)(2 (sxy - mx my) + C2) / ((mx^2 + my^2 + C1)((sxx - mx^2) + (syy - my^2) + C2)).
// Since x enters s(p) only through mx(p), sxx(p) and sxy(p) of the windows that contain it,
//   dSSIM/dx(q) = [G * a](q) + 2 x(q) [G * b](q) + y(q) [G * c](q),
//   a = ds/dmx, b = ds/dsxx, c = ds/dsxy (per pixel, zero outside the image), G symmetric,
// divided by the 3 H W terms of the mean. Four separable passes: horizontal moments, vertical moments +
// per-pixel s / a / b / c (+ the L1 term), horizontal a / b / c, vertical a / b / c + the gradient.
#include <math.h>
#include <string.h>

#include "ngs_internal.cuh"

namespace ngs {
namespace {

constexpr int kRadius = 5;  // 11 taps
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

// The normalised 11-tap Gaussian of sigma 1.5, passed by value (it lands in the constant bank).
struct Window {
  float g[2 * kRadius + 1];
};

// moments per pixel and channel: 5 x 3 planes, [plane][pixel]
__global__ void ssim_hmoments_kernel(Window win, const float* __restrict__ x, const float* __restrict__ y, int W,
                                     int H, float* __restrict__ hm, double* __restrict__ sums) {
  pdl_wait();
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x < 2) sums[threadIdx.x] = 0.0;  // summed by the next kernel
  const int px = blockIdx.x * blockDim.x + threadIdx.x, py = blockIdx.y;
  if (px >= W) return;
  const size_t npix = (size_t)W * H, pix = (size_t)py * W + px;
  float acc[15];
#pragma unroll
  for (int k = 0; k < 15; ++k) acc[k] = 0.f;
  for (int t = -kRadius; t <= kRadius; ++t) {
    const int xx = px + t;
    if (xx < 0 || xx >= W) continue;
    const float g = win.g[t + kRadius];
    const size_t q = (size_t)py * W + xx;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const float a = x[3 * q + ch], b = y[3 * q + ch];
      acc[5 * ch] = fmaf(g, a, acc[5 * ch]);
      acc[5 * ch + 1] = fmaf(g, b, acc[5 * ch + 1]);
      acc[5 * ch + 2] = fmaf(g, a * a, acc[5 * ch + 2]);
      acc[5 * ch + 3] = fmaf(g, b * b, acc[5 * ch + 3]);
      acc[5 * ch + 4] = fmaf(g, a * b, acc[5 * ch + 4]);
    }
  }
#pragma unroll
  for (int k = 0; k < 15; ++k) hm[k * npix + pix] = acc[k];
}

// vertical pass of the moments, the SSIM map and its partials a, b, c (9 planes), the L1 sum and the SSIM
// sum (two doubles, accumulated with one atomic per block)
__global__ void ssim_vmap_kernel(Window win, const float* __restrict__ hm, const float* __restrict__ x,
                                 const float* __restrict__ y, int W, int H, float* __restrict__ abc,
                                 double* __restrict__ sums) {
  pdl_wait();
  const int px = blockIdx.x * blockDim.x + threadIdx.x, py = blockIdx.y;
  const size_t npix = (size_t)W * H;
  float s_sum = 0.f, l1_sum = 0.f;
  if (px < W) {
    const size_t pix = (size_t)py * W + px;
    float m[15];
#pragma unroll
    for (int k = 0; k < 15; ++k) m[k] = 0.f;
    for (int t = -kRadius; t <= kRadius; ++t) {
      const int yy = py + t;
      if (yy < 0 || yy >= H) continue;
      const float g = win.g[t + kRadius];
      const size_t q = (size_t)yy * W + px;
#pragma unroll
      for (int k = 0; k < 15; ++k) m[k] = fmaf(g, hm[k * npix + q], m[k]);
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const float mx = m[5 * ch], my = m[5 * ch + 1], sxx = m[5 * ch + 2], syy = m[5 * ch + 3], sxy = m[5 * ch + 4];
      const float n1 = 2.f * mx * my + kC1, n2 = 2.f * (sxy - mx * my) + kC2;
      const float d1 = mx * mx + my * my + kC1, d2 = (sxx - mx * mx) + (syy - my * my) + kC2;
      const float s = (n1 * n2) / (d1 * d2);
      s_sum += s;
      abc[(3 * ch) * npix + pix] = s * (2.f * my / n1 - 2.f * my / n2 - 2.f * mx / d1 + 2.f * mx / d2);
      abc[(3 * ch + 1) * npix + pix] = -s / d2;
      abc[(3 * ch + 2) * npix + pix] = 2.f * s / n2;
      l1_sum += fabsf(x[3 * pix + ch] - y[3 * pix + ch]);
    }
  }
  // block reduction of the two sums
  __shared__ float r_s[32], r_l[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s_sum += __shfl_xor_sync(0xFFFFFFFFu, s_sum, o);
    l1_sum += __shfl_xor_sync(0xFFFFFFFFu, l1_sum, o);
  }
  if (lane == 0) {
    r_s[warp] = s_sum;
    r_l[warp] = l1_sum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += r_s[w];
      b += r_l[w];
    }
    atomicAdd(&sums[0], a);
    atomicAdd(&sums[1], b);
  }
}

__global__ void ssim_habc_kernel(Window win, const float* __restrict__ abc, int W, int H, float* __restrict__ habc) {
  pdl_wait();
  const int px = blockIdx.x * blockDim.x + threadIdx.x, py = blockIdx.y;
  if (px >= W) return;
  const size_t npix = (size_t)W * H, pix = (size_t)py * W + px;
  float acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.f;
  for (int t = -kRadius; t <= kRadius; ++t) {
    const int xx = px + t;
    if (xx < 0 || xx >= W) continue;
    const float g = win.g[t + kRadius];
    const size_t q = (size_t)py * W + xx;
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = fmaf(g, abc[k * npix + q], acc[k]);
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) habc[k * npix + pix] = acc[k];
}

__global__ void ssim_grad_kernel(Window win, const float* __restrict__ habc, const float* __restrict__ x,
                                 const float* __restrict__ y, int W, int H, float w_l1, float w_ssim,
                                 float* __restrict__ dl) {
  pdl_wait();
  const int px = blockIdx.x * blockDim.x + threadIdx.x, py = blockIdx.y;
  if (px >= W) return;
  const size_t npix = (size_t)W * H, pix = (size_t)py * W + px;
  float acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.f;
  for (int t = -kRadius; t <= kRadius; ++t) {
    const int yy = py + t;
    if (yy < 0 || yy >= H) continue;
    const float g = win.g[t + kRadius];
    const size_t q = (size_t)yy * W + px;
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = fmaf(g, habc[k * npix + q], acc[k]);
  }
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    const float a = x[3 * pix + ch], b = y[3 * pix + ch];
    const float dssim = acc[3 * ch] + 2.f * a * acc[3 * ch + 1] + b * acc[3 * ch + 2];
    const float d = a - b;
    const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
    dl[3 * pix + ch] = w_l1 * sgn - w_ssim * dssim;
  }
}

}  // namespace
}  // namespace ngs

using namespace ngs;

extern "C" NGS_API int ngs_loss_l1_ssim(ngs_ctx* ctx, const float* image, const float* target, int32_t width,
                                        int32_t height, float lambda, float* dl_dimage, double* loss_out,
                                        void* stream) {
  if (!ctx) return NGS_ERR_INVALID_ARG;
  if (!image || !target || width < 1 || height < 1 || width > 16384 || height > 16384 || !(lambda >= 0.f) ||
      !(lambda <= 1.f))
    return fail(ctx, NGS_ERR_INVALID_ARG, "loss: null image/target, size outside 1..16384 or lambda outside [0, 1]");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t npix = (size_t)width * height;
  Window win;
  {
    double g[2 * kRadius + 1], sum = 0.0;
    for (int i = 0; i <= 2 * kRadius; ++i) {
      const double d = (double)(i - kRadius);
      g[i] = exp(-d * d / (2.0 * 1.5 * 1.5));
      sum += g[i];
    }
    for (int i = 0; i <= 2 * kRadius; ++i) win.g[i] = (float)(g[i] / sum);
  }
  const int rc = ensure(ctx, ctx->loss_tmp, sizeof(float) * (15 + 9) * npix + 2 * sizeof(double));
  if (rc != NGS_OK) return rc;
  float* hm = ctx->loss_tmp.as<float>();
  float* abc = hm + 15 * npix;  // 9 planes after the 15 moment planes
  double* sums = reinterpret_cast<double*>(hm + 24 * npix);
  float* habc = hm;  // the moment planes are free again once the map is computed
  const dim3 block(256), grid((width + 255) / 256, height);
  launch_pdl(ssim_hmoments_kernel, grid, block, 0, s, win, image, target, width, height, hm, sums);
  launch_pdl(ssim_vmap_kernel, grid, block, 0, s, win, hm, image, target, width, height, abc, sums);
  int launches = 2;
  if (dl_dimage) {
    const float nterms = 3.f * (float)npix;
    launch_pdl(ssim_habc_kernel, grid, block, 0, s, win, abc, width, height, habc);
    launch_pdl(ssim_grad_kernel, grid, block, 0, s, win, habc, image, target, width, height, (1.f - lambda) / nterms,
               lambda / nterms, dl_dimage);
    launches += 2;
  }
  ctx->launches += launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("loss launch: ") + cudaGetErrorString(e));
  if (loss_out) {  // one synchronisation: the scalar loss to the host (through the mapped mirror)
    publish_words(ctx, reinterpret_cast<const uint64_t*>(sums), 2, kMirrorLoss, s);
    ctx->launches += 1;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(ctx, NGS_ERR_CUDA, std::string("loss read-back: ") + cudaGetErrorString(e));
    const volatile uint64_t* mirror = ctx->h_total + kMirrorLoss;
    const uint64_t w[2] = {mirror[0], mirror[1]};
    double h[2];
    memcpy(h, w, sizeof h);
    const double n = 3.0 * (double)npix;
    loss_out[0] = (1.0 - lambda) * (h[1] / n) + lambda * (1.0 - h[0] / n);
    loss_out[1] = h[1] / n;  // L1
    loss_out[2] = h[0] / n;  // SSIM
  }
  return NGS_OK;
}
