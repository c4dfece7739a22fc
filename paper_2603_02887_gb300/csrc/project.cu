// Projection of 3D Gaussians to splat records (forward) and its adjoint (backward).
//
// Forward (one thread per Gaussian): view transform, EWA screen covariance
// Sigma' = J W R(q) S^2 R(q)^T W^T J^T + dilation I (the 3D Gaussian splatting convention the paper
// builds on, Sec. 3), conic = Sigma'^-1, opacity aleph = sigmoid(logit), emission from real spherical
// harmonics of degree <= 3, the opacity-aware radius r = sqrt(2 ln(aleph / alpha_min) lambda_max(Sigma'))
// outside of which alpha < alpha_min, and the covered tile rectangle.
// Backward: the exact chain rule of the same map, from splat-record gradients to raw parameters.
#include <math.h>

#include <algorithm>

#include "ngs_internal.cuh"

namespace ngs {
namespace {

// Real spherical-harmonic normalisations sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (x sqrt(2) for m != 0).
constexpr float kC0 = 0.28209479177387814f;   // 1 / (2 sqrt(pi))
constexpr float kC1 = 0.4886025119029199f;    // sqrt(3 / (4 pi))
constexpr float kC2a = 1.0925484305920792f;   // sqrt(15 / (4 pi))
constexpr float kC2b = 0.31539156525252005f;  // sqrt(5 / (16 pi))
constexpr float kC2c = 0.5462742152960396f;   // sqrt(15 / (16 pi))
constexpr float kC3a = 0.5900435899266435f;   // sqrt(35 / (32 pi))
constexpr float kC3b = 2.890611442640554f;    // sqrt(105 / (4 pi))
constexpr float kC3c = 0.4570457994644658f;   // sqrt(21 / (32 pi))
constexpr float kC3d = 0.3731763325901154f;   // sqrt(7 / (16 pi))
constexpr float kC3e = 1.445305721320277f;    // sqrt(105 / (16 pi))

// Basis in the coefficient order and sign convention of 3D Gaussian splatting assets.
__device__ __forceinline__ void sh_basis(int degree, float x, float y, float z, float* Y) {
  Y[0] = kC0;
  if (degree < 1) return;
  Y[1] = -kC1 * y;
  Y[2] = kC1 * z;
  Y[3] = -kC1 * x;
  if (degree < 2) return;
  float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kC2a * x * y;
  Y[5] = -kC2a * y * z;
  Y[6] = kC2b * (2.f * zz - xx - yy);
  Y[7] = -kC2a * x * z;
  Y[8] = kC2c * (xx - yy);
  if (degree < 3) return;
  Y[9] = -kC3a * y * (3.f * xx - yy);
  Y[10] = kC3b * x * y * z;
  Y[11] = -kC3c * y * (4.f * zz - xx - yy);
  Y[12] = kC3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = -kC3c * x * (4.f * zz - xx - yy);
  Y[14] = kC3e * z * (xx - yy);
  Y[15] = -kC3a * x * (xx - 3.f * yy);
}

// sum_k w_k grad Y_k(x, y, z), treating (x, y, z) as free variables.
__device__ __forceinline__ void sh_basis_grad(int degree, float x, float y, float z, const float* w, float& gx,
                                              float& gy, float& gz) {
  gx = gy = gz = 0.f;
  if (degree < 1) return;
  gy += -kC1 * w[1];
  gz += kC1 * w[2];
  gx += -kC1 * w[3];
  if (degree < 2) return;
  float xx = x * x, yy = y * y, zz = z * z;
  gx += kC2a * y * w[4];
  gy += kC2a * x * w[4];
  gy += -kC2a * z * w[5];
  gz += -kC2a * y * w[5];
  gx += -2.f * kC2b * x * w[6];
  gy += -2.f * kC2b * y * w[6];
  gz += 4.f * kC2b * z * w[6];
  gx += -kC2a * z * w[7];
  gz += -kC2a * x * w[7];
  gx += 2.f * kC2c * x * w[8];
  gy += -2.f * kC2c * y * w[8];
  if (degree < 3) return;
  gx += -6.f * kC3a * x * y * w[9];
  gy += -kC3a * (3.f * xx - 3.f * yy) * w[9];
  gx += kC3b * y * z * w[10];
  gy += kC3b * x * z * w[10];
  gz += kC3b * x * y * w[10];
  gx += 2.f * kC3c * x * y * w[11];
  gy += -kC3c * (4.f * zz - xx - 3.f * yy) * w[11];
  gz += -8.f * kC3c * y * z * w[11];
  gx += -6.f * kC3d * x * z * w[12];
  gy += -6.f * kC3d * y * z * w[12];
  gz += kC3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
  gx += -kC3c * (4.f * zz - 3.f * xx - yy) * w[13];
  gy += 2.f * kC3c * x * y * w[13];
  gz += -8.f * kC3c * x * z * w[13];
  gx += 2.f * kC3e * x * z * w[14];
  gy += -2.f * kC3e * y * z * w[14];
  gz += kC3e * (xx - yy) * w[14];
  gx += -kC3a * (3.f * xx - 3.f * yy) * w[15];
  gy += 6.f * kC3a * x * y * w[15];
}

// FP32 view depth with a fixed fma order (the sort key; also used for the near-plane test).
__device__ __forceinline__ float view_depth(const CamParams& c, float px, float py, float pz) {
  float z = __fmaf_rn(c.R[6], px, c.t[2]);
  z = __fmaf_rn(c.R[7], py, z);
  return __fmaf_rn(c.R[8], pz, z);
}

__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float* R) {
  R[0] = 1.f - 2.f * (y * y + z * z);
  R[1] = 2.f * (x * y - w * z);
  R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);
  R[4] = 1.f - 2.f * (x * x + z * z);
  R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);
  R[7] = 2.f * (y * z + w * x);
  R[8] = 1.f - 2.f * (x * x + y * y);
}

// Everything the forward map computes that the backward needs again.
template <int DEG>
struct ProjState {
  static constexpr int K = (DEG + 1) * (DEG + 1);
  float x, y, z, iz;       // view-space mean, 1/z
  float qn[4], qnorm;      // normalised quaternion and the raw norm
  float Rq[9], S[3];       // rotation and scales
  float M[9];              // Rq diag(S)
  float T[6];              // J W
  float U[6];              // T M: column i is the projected axis i, S_i T Rq e_i
  float s00, s01, s11;     // 2D covariance U U^T + dilation I
  float det;               // its determinant
  float A, B, C;           // conic
  float aleph;
  float dir[3], dnorm;     // unit direction from the camera centre, |p - campos|
  float e[3];              // unclamped emission
  float Y[K];
};

// SH coefficients of Gaussian i: 3K floats. VEC: the block starts on a 16-byte boundary and 3K is a multiple
// of 4 (degree 1 or 3 with an aligned base), so it is read with 16-byte loads.
template <int K, bool VEC>
__device__ __forceinline__ void load_sh(const float* sh, float (&c)[3 * K]) {
  if constexpr (VEC) {
    const float4* p = reinterpret_cast<const float4*>(sh);
#pragma unroll
    for (int k = 0; k < 3 * K / 4; ++k) {
      float4 t = p[k];
      c[4 * k] = t.x;
      c[4 * k + 1] = t.y;
      c[4 * k + 2] = t.z;
      c[4 * k + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 3 * K; ++k) c[k] = sh[k];
  }
}

template <int K, bool VEC>
__device__ __forceinline__ void store_sh(float* dst, const float (&c)[3 * K]) {
  if constexpr (VEC) {
#pragma unroll
    for (int k = 0; k < 3 * K / 4; ++k)
      reinterpret_cast<float4*>(dst)[k] = make_float4(c[4 * k], c[4 * k + 1], c[4 * k + 2], c[4 * k + 3]);
  } else {
#pragma unroll
    for (int k = 0; k < 3 * K; ++k) dst[k] = c[k];
  }
}

// A request to bring the line holding `p` into L1 (PTX prefetch; no register is written).
__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// The raw parameters of one Gaussian other than its SH coefficients, read in one go so that their loads
// are in flight together (the quaternion as one 16-byte load when the array is 16-byte aligned).
struct RawParams {
  float m[3], ls[3], q[4], logit;
};

__device__ __forceinline__ RawParams load_params(const ngs_gaussians& g, int i) {
  RawParams r;
  const float* m = g.means + 3 * (int64_t)i;
  const float* ls = g.log_scales + 3 * (int64_t)i;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r.m[k] = m[k];
    r.ls[k] = ls[k];
  }
  if (((uintptr_t)g.quats & 15) == 0) {
    const float4 q = reinterpret_cast<const float4*>(g.quats)[i];
    r.q[0] = q.x, r.q[1] = q.y, r.q[2] = q.z, r.q[3] = q.w;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) r.q[k] = g.quats[4 * (int64_t)i + k];
  }
  r.logit = g.opacity_logits[i];
  return r;
}

// sh_src: Gaussian i's 3K SH coefficients (in global memory, or staged in shared memory by the caller).
template <int DEG, bool VEC = false>
__device__ __forceinline__ void forward_map(const RawParams& prm, const CamParams& cam, const RenderParams& rp,
                                            ProjState<DEG>& st, const float* sh_src) {
  constexpr int K = ProjState<DEG>::K;
  const float px = prm.m[0], py = prm.m[1], pz = prm.m[2];
  st.x = cam.R[0] * px + cam.R[1] * py + cam.R[2] * pz + cam.t[0];
  st.y = cam.R[3] * px + cam.R[4] * py + cam.R[5] * pz + cam.t[1];
  st.z = view_depth(cam, px, py, pz);
  st.iz = 1.f / st.z;
  const float* q = prm.q;
  st.qnorm = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  float inv = 1.f / st.qnorm;
#pragma unroll
  for (int k = 0; k < 4; ++k) st.qn[k] = q[k] * inv;
  quat_to_rot(st.qn[0], st.qn[1], st.qn[2], st.qn[3], st.Rq);
#pragma unroll
  for (int k = 0; k < 3; ++k) st.S[k] = expf(prm.ls[k]);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) st.M[3 * r + c] = st.Rq[3 * r + c] * st.S[c];
  float j00 = cam.fx * st.iz, j02 = -cam.fx * st.x * st.iz * st.iz;
  float j11 = cam.fy * st.iz, j12 = -cam.fy * st.y * st.iz * st.iz;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    st.T[c] = j00 * cam.R[c] + j02 * cam.R[6 + c];
    st.T[3 + c] = j11 * cam.R[3 + c] + j12 * cam.R[6 + c];
  }
  // projected axes U = T M; Sigma' = U U^T + dilation I. Its determinant by Cauchy-Binet,
  // det = sum_{i<j} (u_i x u_j)^2 + dilation tr(U U^T) + dilation^2, has no cancellation when the splat is
  // a thin needle (det(Sigma') as s00 s11 - s01^2 would lose most of its digits).
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    st.U[c] = st.T[0] * st.M[c] + st.T[1] * st.M[3 + c] + st.T[2] * st.M[6 + c];
    st.U[3 + c] = st.T[3] * st.M[c] + st.T[4] * st.M[3 + c] + st.T[5] * st.M[6 + c];
  }
  float t00 = st.U[0] * st.U[0] + st.U[1] * st.U[1] + st.U[2] * st.U[2];
  float t11 = st.U[3] * st.U[3] + st.U[4] * st.U[4] + st.U[5] * st.U[5];
  st.s00 = t00 + rp.dilation;
  st.s01 = st.U[0] * st.U[3] + st.U[1] * st.U[4] + st.U[2] * st.U[5];
  st.s11 = t11 + rp.dilation;
  float m01 = st.U[0] * st.U[4] - st.U[1] * st.U[3];
  float m02 = st.U[0] * st.U[5] - st.U[2] * st.U[3];
  float m12 = st.U[1] * st.U[5] - st.U[2] * st.U[4];
  st.det = m01 * m01 + m02 * m02 + m12 * m12 + rp.dilation * (t00 + t11) + rp.dilation * rp.dilation;
  float idet = 1.f / st.det;
  st.A = st.s11 * idet;
  st.B = -st.s01 * idet;
  st.C = st.s00 * idet;
  st.aleph = 1.f / (1.f + expf(-prm.logit));
  float d0 = px - cam.campos[0], d1 = py - cam.campos[1], d2 = pz - cam.campos[2];
  st.dnorm = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  float idn = 1.f / st.dnorm;
  st.dir[0] = d0 * idn;
  st.dir[1] = d1 * idn;
  st.dir[2] = d2 * idn;
  sh_basis(DEG, st.dir[0], st.dir[1], st.dir[2], st.Y);
  float sh[3 * K];
  load_sh<K, VEC>(sh_src, sh);
  float e0 = 0.5f, e1 = 0.5f, e2 = 0.5f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    e0 += st.Y[k] * sh[3 * k];
    e1 += st.Y[k] * sh[3 * k + 1];
    e2 += st.Y[k] * sh[3 * k + 2];
  }
  st.e[0] = e0;
  st.e[1] = e1;
  st.e[2] = e2;
}

// ---- tile binning --------------------------------------------------------------------------------
// A splat reaches pixel p iff L + q'(p - mu) >= log2(alpha_min), q'(d) = A' dx^2 + B' dx dy + C' dy^2 the
// concave exponent of the record (the compositing kernels' test). Binning keeps the ellipse
// q'(d) >= Tm = T' - (0.01 + 0.001 |T'|), T' = log2(alpha_min) - L (a margin over the per-pixel test), and
// for every tile row of its bounding box takes the tiles that the ellipse's x-extent over the row's band of
// pixel centres reaches. Along the band the right boundary of the ellipse is concave in dy, so its maximum
// sits at the ellipse's rightmost point clamped to the band (the left boundary is convex: minimum at the
// clamped leftmost point, its mirror image). Every operation is one FP32 rounding in a fixed order, so the
// count (projection), the emission and the tile-binning oracle agree.
struct SplatBin {
  float u, v, A, B, C, Tm;
  float dymax, dyr;  // half height of the ellipse; dy of its rightmost point
};

__device__ __forceinline__ SplatBin splat_bin(float4 r0, float4 r1, float log2_amin) {
  SplatBin b;
  b.u = r0.x;
  b.v = r0.y;
  b.A = r0.z;
  b.B = r0.w;
  b.C = r1.x;
  float Tp = __fsub_rn(log2_amin, r1.y);
  b.Tm = __fsub_rn(Tp, __fadd_rn(0.01f, __fmul_rn(0.001f, fabsf(Tp))));
  // delta = 4 A' C' - B'^2 > 0; the ellipse spans |dy| <= sqrt(4 A' Tm / delta), |dx| <= sqrt(4 C' Tm / delta)
  float delta = __fsub_rn(__fmul_rn(__fmul_rn(4.0f, b.A), b.C), __fmul_rn(b.B, b.B));
  float four_tm = __fmul_rn(4.0f, b.Tm);
  b.dymax = __fsqrt_rn(fmaxf(__fdiv_rn(__fmul_rn(four_tm, b.A), delta), 0.0f));
  float dxmax = __fsqrt_rn(fmaxf(__fdiv_rn(__fmul_rn(four_tm, b.C), delta), 0.0f));
  b.dyr = -__fdiv_rn(__fmul_rn(b.B, dxmax), __fmul_rn(2.0f, b.C));
  return b;
}

// Roots in dx of A' dx^2 + (B' t) dx + (C' t^2 - Tm) = 0 at height t (A' < 0): left (sign = +1) and right
// (sign = -1) boundary of the ellipse.
__device__ __forceinline__ float ellipse_x(const SplatBin& b, float t, float sign) {
  float Bt = __fmul_rn(b.B, t);
  float D = __fsub_rn(__fmul_rn(Bt, Bt), __fmul_rn(__fmul_rn(4.0f, b.A), __fsub_rn(__fmul_rn(__fmul_rn(b.C, t), t), b.Tm)));
  float r = __fsqrt_rn(fmaxf(D, 0.0f));
  return __fdiv_rn(__fadd_rn(-Bt, __fmul_rn(sign, r)), __fmul_rn(2.0f, b.A));
}

// Tile columns [tx0, tx1] of tile row ty reached by the ellipse, clipped to [x0, x1]; false if none.
__device__ __forceinline__ bool row_span(const SplatBin& b, const RenderParams& rp, int ty, int x0, int x1, int& tx0,
                                         int& tx1) {
  float a = __fsub_rn((float)(ty * rp.tile_h) + 0.5f, b.v);
  float c = __fsub_rn((float)(ty * rp.tile_h + rp.tile_h) - 0.5f, b.v);
  a = fmaxf(a, -b.dymax);
  c = fminf(c, b.dymax);
  if (!(a <= c)) return false;
  float xl = ellipse_x(b, fminf(fmaxf(-b.dyr, a), c), 1.0f);
  float xr = ellipse_x(b, fminf(fmaxf(b.dyr, a), c), -1.0f);
  float itw = 1.0f / (float)rp.tile_w;  // power of two: exact
  float f0 = floorf(__fmul_rn(__fsub_rn(__fadd_rn(b.u, xl), 0.5f), itw));
  float f1 = floorf(__fmul_rn(__fsub_rn(__fadd_rn(b.u, xr), 0.5f), itw));
  if (!(f0 <= (float)x1 && f1 >= (float)x0)) return false;
  tx0 = (int)fmaxf(f0, (float)x0);
  tx1 = (int)fminf(f1, (float)x1);
  return tx0 <= tx1;
}

// Tile bounding box of the splat (u, v) with half extents (rx, ry): identical arithmetic everywhere.
__device__ __forceinline__ bool tile_rect(float u, float v, float rx, float ry, const RenderParams& rp, int& x0,
                                          int& x1, int& y0, int& y1) {
  float itw = 1.0f / (float)rp.tile_w, ith = 1.0f / (float)rp.tile_h;  // powers of two: exact
  float fx0 = floorf(__fmul_rn(__fsub_rn(__fsub_rn(u, rx), 0.5f), itw));
  float fx1 = floorf(__fmul_rn(__fsub_rn(__fadd_rn(u, rx), 0.5f), itw));
  float fy0 = floorf(__fmul_rn(__fsub_rn(__fsub_rn(v, ry), 0.5f), ith));
  float fy1 = floorf(__fmul_rn(__fsub_rn(__fadd_rn(v, ry), 0.5f), ith));
  bool ok = rx > 0.f && ry > 0.f && fx1 >= 0.f && fx0 <= (float)(rp.tiles_x - 1) && fy1 >= 0.f &&
            fy0 <= (float)(rp.tiles_y - 1) && isfinite(fx0) && isfinite(fx1) && isfinite(fy0) && isfinite(fy1);
  if (!ok) return false;
  x0 = (int)fmaxf(fx0, 0.f);
  x1 = (int)fminf(fx1, (float)(rp.tiles_x - 1));
  y0 = (int)fmaxf(fy0, 0.f);
  y1 = (int)fminf(fy1, (float)(rp.tiles_y - 1));
  return true;
}

// Tiles covered over tile rows [y0, y1] (columns clipped to [x0, x1]).
__device__ __forceinline__ uint32_t count_rows(const SplatBin& b, const RenderParams& rp, int x0, int x1, int y0,
                                               int y1) {
  uint32_t c = 0;
  for (int ty = y0; ty <= y1; ++ty) {
    int t0, t1;
    if (row_span(b, rp, ty, x0, x1, t0, t1)) c += (uint32_t)(t1 - t0 + 1);
  }
  return c;
}

// A splat spanning more tile rows than this has them counted by its whole warp, one row per lane.
constexpr int kCoopRows = 8;

// Block b works on view b % n_views and Gaussians [256 (b / n_views), +256): the views of one block of
// Gaussians run side by side, so their parameters are read from HBM once and from L2 afterwards.
// A single view takes its camera from the kernel parameters (cam0), a batch (or a captured graph, which
// must serve any pose) from the view table; the arithmetic below is the same code either way.
template <int DEG, bool VEC>
__global__ void __launch_bounds__(256, 4) project_kernel(ngs_gaussians g, const ViewParams* __restrict__ views,
                                                      CamParams cam0, RenderParams rp, float4* rec,
                                                      uint32_t* depth_key, uint32_t* tile_count, uint32_t* order) {
  pdl_wait();
  const uint32_t view = blockIdx.x % rp.n_views;
  const int i = (blockIdx.x / rp.n_views) * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  if (rp.n_views != 1) {  // the block's view (one per block)
    rp.tiles_x = views[view].tiles_x;
    rp.tiles_y = views[view].tiles_y;
  }
  const int64_t r = (int64_t)view * g.n + i;  // record index
  if (i < g.n) {
    // every line the projection reads, requested at once: the loads behind the depth test and inside the
    // colour find them in L1 instead of making three round trips to memory one after another
    prefetch_l1(g.means + 3 * (int64_t)i);
    prefetch_l1(g.log_scales + 3 * (int64_t)i);
    prefetch_l1(g.quats + 4 * (int64_t)i);
    prefetch_l1(g.opacity_logits + i);
    const char* sh = reinterpret_cast<const char*>(g.sh + (int64_t)i * ProjState<DEG>::K * 3);
    constexpr int kShBytes = ProjState<DEG>::K * 3 * 4;
#pragma unroll
    for (int o = 0; o < kShBytes; o += 128) prefetch_l1(sh + o);
    prefetch_l1(sh + kShBytes - 4);
  }
  // every lane stays to the end: the warp counts its tall splats' tiles together
  uint32_t count = 0;
  bool tall = false;
  int x0 = 0, x1 = -1, y0 = 0, y1 = -1;
  SplatBin b = {};
  float z = 0.f;
  if (i < g.n) {
    const CamParams cam = rp.cam_from_table ? views[view].cam : cam0;
    const float* m = g.means + 3 * (int64_t)i;
    z = view_depth(cam, m[0], m[1], m[2]);
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = make_float4(0.f, z, 0.f, 0.f);
    if (z > rp.near_plane) {
      ProjState<DEG> st;
      forward_map<DEG, VEC>(load_params(g, i), cam, rp, st, g.sh + (int64_t)i * ProjState<DEG>::K * 3);
      if (st.det > 0.f && st.aleph >= rp.alpha_min && isfinite(st.A) && isfinite(st.C)) {
        float u = cam.fx * st.x * st.iz + cam.cx;
        float v = cam.fy * st.y * st.iz + cam.cy;
        float L = log2f(st.aleph);
        // alpha >= alpha_min needs d^T conic d <= tau = 2 ln(aleph/alpha_min): an ellipse whose bounding box
        // has half extents sqrt(tau s00), sqrt(tau s11); widened by 1e-4 relative and one pixel so that FP32
        // rounding never cuts a pixel
        float tau = fmaxf(2.f * kLn2 * (L - rp.log2_alpha_min), 0.f);
        float rx = sqrtf(tau * st.s00) * 1.0001f + 1.0f;
        float ry = sqrtf(tau * st.s11) * 1.0001f + 1.0f;
        float E0 = fmaxf(st.e[0], 0.f), E1 = fmaxf(st.e[1], 0.f), E2 = fmaxf(st.e[2], 0.f);
        r0 = make_float4(u, v, kConicScale * st.A, 2.f * kConicScale * st.B);
        r1 = make_float4(kConicScale * st.C, L, E0, E1);
        r2 = make_float4(E2, z, rx, ry);
        if (tile_rect(r0.x, r0.y, r2.z, r2.w, rp, x0, x1, y0, y1)) {
          b = splat_bin(r0, r1, rp.log2_alpha_min);
          tall = y1 - y0 >= kCoopRows;
          if (!tall) count = count_rows(b, rp, x0, x1, y0, y1);
        }
      }
    }
    rec[3 * r] = r0;
    rec[3 * r + 1] = r1;
    rec[3 * r + 2] = r2;
    order[r] = (uint32_t)r;
  }
  // tall splats, one after another: lane l counts tile rows y0 + l, y0 + l + 32, ... (the same row spans)
  for (uint32_t pending = __ballot_sync(0xFFFFFFFFu, tall); pending != 0u; pending &= pending - 1u) {
    const int src = __ffs(pending) - 1;
    SplatBin cb;
    cb.u = __shfl_sync(0xFFFFFFFFu, b.u, src);
    cb.v = __shfl_sync(0xFFFFFFFFu, b.v, src);
    cb.A = __shfl_sync(0xFFFFFFFFu, b.A, src);
    cb.B = __shfl_sync(0xFFFFFFFFu, b.B, src);
    cb.C = __shfl_sync(0xFFFFFFFFu, b.C, src);
    cb.Tm = __shfl_sync(0xFFFFFFFFu, b.Tm, src);
    cb.dymax = __shfl_sync(0xFFFFFFFFu, b.dymax, src);
    cb.dyr = __shfl_sync(0xFFFFFFFFu, b.dyr, src);
    const int cx0 = __shfl_sync(0xFFFFFFFFu, x0, src), cx1 = __shfl_sync(0xFFFFFFFFu, x1, src);
    const int cy0 = __shfl_sync(0xFFFFFFFFu, y0, src), cy1 = __shfl_sync(0xFFFFFFFFu, y1, src);
    uint32_t c = 0;
    for (int ty = cy0 + lane; ty <= cy1; ty += 32) {
      int t0, t1;
      if (row_span(cb, rp, ty, cx0, cx1, t0, t1)) c += (uint32_t)(t1 - t0 + 1);
    }
    c = __reduce_add_sync(0xFFFFFFFFu, c);
    if (lane == src) count = c;
  }
  if (i < g.n) {
    depth_key[r] = count ? __float_as_uint(z) : 0xFFFFFFFFu;
    tile_count[r] = count;
  }
}

// A record with more pairs than this is emitted by its whole warp, one tile row per lane; smaller ones by
// their own lane. One thread per record would leave a warp waiting on its largest splat: a few splats near
// the camera cover hundreds of tiles while most cover a handful (SIMT efficiency 0.40 measured on GB300
// at 500k / 1080p on 8x8 tiles).
constexpr uint32_t kCoopPairs = 32;

__global__ void __launch_bounds__(256) emit_pairs_kernel(const float4* rec, const uint32_t* order,
                                                         const uint32_t* offsets, const ViewParams* __restrict__ views,
                                                         RenderParams rp, uint32_t* tiles, uint32_t* vals,
                                                         uint32_t cap) {
  pdl_wait();
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  // every lane stays to the end: the warp emits its large records together
  uint32_t off = 0, end = 0, id = 0;
  int x0 = 0, x1 = -1, y0 = 0, y1 = -1, tiles_x = 0;
  SplatBin b = {};
  bool live = false;
  if (s < rp.n_records) {
    off = offsets[s];
    end = min(offsets[s + 1], cap);  // slots past the capacity are not written
    if (off < end) {
      id = order[s];
      const uint32_t view = id / rp.n_gaussians;
      RenderParams rv = rp;
      rv.tiles_x = views[view].tiles_x;
      rv.tiles_y = views[view].tiles_y;
      const float4 r0 = rec[3 * (int64_t)id], r1 = rec[3 * (int64_t)id + 1], r2 = rec[3 * (int64_t)id + 2];
      if (tile_rect(r0.x, r0.y, r2.z, r2.w, rv, x0, x1, y0, y1)) {
        b = splat_bin(r0, r1, rp.log2_alpha_min);
        tiles_x = rv.tiles_x;
        live = true;
      }
    }
  }
  const bool coop = live && end - off > kCoopPairs;
  if (live && !coop) {
    for (int ty = y0; ty <= y1 && off < end; ++ty) {
      int t0, t1;
      if (!row_span(b, rp, ty, x0, x1, t0, t1)) continue;
      uint32_t tile = (uint32_t)(ty * tiles_x + t0);  // within the view
      for (int tx = t0; tx <= t1 && off < end; ++tx, ++tile, ++off) {
        tiles[off] = tile;
        vals[off] = id;
      }
    }
  }
  // the warp's large records, one after another: lane l takes tile rows y0 + l, y0 + l + 32, ...; a warp
  // prefix sum of the rows' span lengths gives each row its slots, so the pairs land exactly where one
  // thread walking the rows in order would put them
  for (uint32_t pending = __ballot_sync(0xFFFFFFFFu, coop); pending != 0u; pending &= pending - 1u) {
    const int src = __ffs(pending) - 1;
    SplatBin cb;
    cb.u = __shfl_sync(0xFFFFFFFFu, b.u, src);
    cb.v = __shfl_sync(0xFFFFFFFFu, b.v, src);
    cb.A = __shfl_sync(0xFFFFFFFFu, b.A, src);
    cb.B = __shfl_sync(0xFFFFFFFFu, b.B, src);
    cb.C = __shfl_sync(0xFFFFFFFFu, b.C, src);
    cb.Tm = __shfl_sync(0xFFFFFFFFu, b.Tm, src);
    cb.dymax = __shfl_sync(0xFFFFFFFFu, b.dymax, src);
    cb.dyr = __shfl_sync(0xFFFFFFFFu, b.dyr, src);
    const int cx0 = __shfl_sync(0xFFFFFFFFu, x0, src), cx1 = __shfl_sync(0xFFFFFFFFu, x1, src);
    const int cy0 = __shfl_sync(0xFFFFFFFFu, y0, src), cy1 = __shfl_sync(0xFFFFFFFFu, y1, src);
    const int ctx = __shfl_sync(0xFFFFFFFFu, tiles_x, src);
    const uint32_t cid = __shfl_sync(0xFFFFFFFFu, id, src), cend = __shfl_sync(0xFFFFFFFFu, end, src);
    uint32_t coff = __shfl_sync(0xFFFFFFFFu, off, src);
    for (int ty0 = cy0; ty0 <= cy1 && coff < cend; ty0 += 32) {
      const int ty = ty0 + lane;
      int t0 = 0, t1 = -1;
      const bool has = ty <= cy1 && row_span(cb, rp, ty, cx0, cx1, t0, t1);
      const uint32_t len = has ? (uint32_t)(t1 - t0 + 1) : 0u;
      uint32_t incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
      }
      uint32_t o = coff + incl - len;
      uint32_t tile = (uint32_t)(ty * ctx + t0);
      for (int tx = t0; tx <= t1 && o < cend; ++tx, ++tile, ++o) {
        tiles[o] = tile;
        vals[o] = cid;
      }
      coff += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
  }
}

// Gradient of the loss w.r.t. one Gaussian's raw parameters, summed over views.
template <int DEG>
struct ParamGrad {
  static constexpr int K = (DEG + 1) * (DEG + 1);
  float m[3], ls[3], q[4], op, sh[3 * K];
};

// Adds view `cam`'s share of Gaussian i's parameter gradient (from its splat-record gradient `gr`) to acc.
// DIRECT (a single view): each gradient is stored to `out` as soon as it is known instead, which keeps it
// out of the registers live across the rest of the chain.
template <int DEG, bool VEC, bool DIRECT>
__device__ __forceinline__ void add_view_gradient(const RawParams& prm, const CamParams& cam,
                                                  const RenderParams& rp, int i, float4 g0, float4 g1, float4 g2,
                                                  ParamGrad<DEG>& acc, const ngs_grads& out, const float* sh_src,
                                                  float* dsh_dst) {
  constexpr int K = ProjState<DEG>::K;
  // the replay accumulates w / ln 2 (w = dL/d(log2 alpha)): restore the factor on the six moments
  g0 = make_float4(g0.x * kLn2, g0.y * kLn2, g0.z * kLn2, g0.w * kLn2);
  g1.x *= kLn2;
  g1.y *= kLn2;
  ProjState<DEG> st;
  forward_map<DEG, VEC>(prm, cam, rp, st, sh_src);
  // moments -> record gradient (the record's A', B', C' are these same products) -> natural quantities
  const float Ap = kConicScale * st.A, Bp = 2.f * kConicScale * st.B, Cp = kConicScale * st.C;
  float du = -(2.f * Ap * g0.x + Bp * g0.y);
  float dv = -(Bp * g0.x + 2.f * Cp * g0.y);
  float dA = g0.z * kConicScale, dB = g0.w * 2.f * kConicScale, dC = g1.x * kConicScale;
  float dE[3] = {g1.z, g1.w, g2.x};
  const float gop = g1.y * (1.f - st.aleph) / kLn2;  // L = log2(sigmoid(logit))
  if constexpr (DIRECT) out.d_opacity_logits[i] = gop;
  else acc.op += gop;
  // conic Q = Sigma'^-1 with Sigma' = U U^T + dilation I: dLoss/dSigma' = -Q G Q, G = [[dA, dB/2], [dB/2, dC]].
  // Every term of the chain is needed only as Hs u_i = -Q G Q u_i for the projected axes u_i (columns of U):
  //   dLoss/dM (column i) = 2 T^T Hs u_i,   dLoss/dT = 2 sum_i (Hs u_i) M_i^T.
  // Q u_i is formed by Sherman-Morrison from R_i = Sigma' - u_i u_i^T (the other two axes plus dilation):
  //   Q u_i = R_i^-1 u_i / (1 + u_i^T R_i^-1 u_i),
  // which stays accurate for thin needles, where Q u_i along the long axis is a small difference of large
  // terms if formed directly.
  const float dil = rp.dilation;
  const float hG01 = 0.5f * dB;
  float HU[6];  // [2][3]: Hs u_i
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int j = ax == 0 ? 1 : 0, k = ax == 2 ? 1 : 2;
    const float ui0 = st.U[ax], ui1 = st.U[3 + ax];
    const float uj0 = st.U[j], uj1 = st.U[3 + j], uk0 = st.U[k], uk1 = st.U[3 + k];
    const float r00 = uj0 * uj0 + uk0 * uk0 + dil, r01 = uj0 * uj1 + uk0 * uk1, r11 = uj1 * uj1 + uk1 * uk1 + dil;
    const float mjk = uj0 * uk1 - uk0 * uj1;
    const float detR = mjk * mjk + dil * (uj0 * uj0 + uj1 * uj1 + uk0 * uk0 + uk1 * uk1) + dil * dil;
    const float a0 = (r11 * ui0 - r01 * ui1) / detR, a1 = (r00 * ui1 - r01 * ui0) / detR;
    const float den = 1.f + ui0 * a0 + ui1 * a1;
    const float q0 = a0 / den, q1 = a1 / den;           // Q u_i
    const float g0 = dA * q0 + hG01 * q1, g1 = hG01 * q0 + dC * q1;  // G Q u_i
    HU[ax] = -(st.A * g0 + st.B * g1);
    HU[3 + ax] = -(st.B * g0 + st.C * g1);
  }
  float dM[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) dM[3 * r + c] = 2.f * (st.T[r] * HU[c] + st.T[3 + r] * HU[3 + c]);
  float dT[6];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      dT[3 * a + c] = 2.f * (HU[3 * a] * st.M[3 * c] + HU[3 * a + 1] * st.M[3 * c + 1] + HU[3 * a + 2] * st.M[3 * c + 2]);
  // T = J W: dJ = dT W^T (only the four nonzero entries of J)
  float dJ00 = dT[0] * cam.R[0] + dT[1] * cam.R[1] + dT[2] * cam.R[2];
  float dJ02 = dT[0] * cam.R[6] + dT[1] * cam.R[7] + dT[2] * cam.R[8];
  float dJ11 = dT[3] * cam.R[3] + dT[4] * cam.R[4] + dT[5] * cam.R[5];
  float dJ12 = dT[3] * cam.R[6] + dT[4] * cam.R[7] + dT[5] * cam.R[8];
  float iz = st.iz, iz2 = iz * iz, iz3 = iz2 * iz;
  float dvx = du * cam.fx * iz - dJ02 * cam.fx * iz2;
  float dvy = dv * cam.fy * iz - dJ12 * cam.fy * iz2;
  float dvz = -du * cam.fx * st.x * iz2 - dv * cam.fy * st.y * iz2 - dJ00 * cam.fx * iz2 +
              dJ02 * 2.f * cam.fx * st.x * iz3 - dJ11 * cam.fy * iz2 + dJ12 * 2.f * cam.fy * st.y * iz3;
  float gm[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) gm[c] = cam.R[c] * dvx + cam.R[3 + c] * dvy + cam.R[6 + c] * dvz;
  // M = Rq diag(S)
  float dRq[9], dS[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      dRq[3 * r + c] = dM[3 * r + c] * st.S[c];
      dS[c] += dM[3 * r + c] * st.Rq[3 * r + c];
    }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (DIRECT) out.d_log_scales[3 * (int64_t)i + c] = dS[c] * st.S[c];
    else acc.ls[c] += dS[c] * st.S[c];
  }
  // rotation matrix of the unit quaternion (w, a, b, c)
  float w = st.qn[0], a = st.qn[1], b = st.qn[2], c = st.qn[3];
  const float* D = dRq;
  float dqn[4];
  dqn[0] = 2.f * (-c * D[1] + b * D[2] + c * D[3] - a * D[5] - b * D[6] + a * D[7]);
  dqn[1] = 2.f * (b * D[1] + c * D[2] + b * D[3] - 2.f * a * D[4] - w * D[5] + c * D[6] + w * D[7] - 2.f * a * D[8]);
  dqn[2] = 2.f * (-2.f * b * D[0] + a * D[1] + w * D[2] + a * D[3] + c * D[5] - w * D[6] + c * D[7] - 2.f * b * D[8]);
  dqn[3] = 2.f * (-2.f * c * D[0] - w * D[1] + a * D[2] + w * D[3] - 2.f * c * D[4] + b * D[5] + a * D[6] + b * D[7]);
  float dot = st.qn[0] * dqn[0] + st.qn[1] * dqn[1] + st.qn[2] * dqn[2] + st.qn[3] * dqn[3];
  float iq = 1.f / st.qnorm;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if constexpr (DIRECT) out.d_quats[4 * (int64_t)i + k] = (dqn[k] - st.qn[k] * dot) * iq;
    else acc.q[k] += (dqn[k] - st.qn[k] * dot) * iq;
  }
  // emission: dE/dsh = Y (unclamped channels); direction term into the mean
  float sh[3 * K];
  load_sh<K, VEC>(sh_src, sh);
  float d0 = st.e[0] < 0.f ? 0.f : dE[0];
  float d1 = st.e[1] < 0.f ? 0.f : dE[1];
  float d2 = st.e[2] < 0.f ? 0.f : dE[2];
  float wk[K];
#pragma unroll
  for (int k = 0; k < K; ++k) wk[k] = d0 * sh[3 * k] + d1 * sh[3 * k + 1] + d2 * sh[3 * k + 2];
  if constexpr (DIRECT) {
    float gsh[3 * K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      gsh[3 * k] = d0 * st.Y[k];
      gsh[3 * k + 1] = d1 * st.Y[k];
      gsh[3 * k + 2] = d2 * st.Y[k];
    }
    store_sh<K, VEC>(dsh_dst, gsh);
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      acc.sh[3 * k] += d0 * st.Y[k];
      acc.sh[3 * k + 1] += d1 * st.Y[k];
      acc.sh[3 * k + 2] += d2 * st.Y[k];
    }
  }
  float gdx, gdy, gdz;
  sh_basis_grad(DEG, st.dir[0], st.dir[1], st.dir[2], wk, gdx, gdy, gdz);
  float rad = st.dir[0] * gdx + st.dir[1] * gdy + st.dir[2] * gdz;
  float idn = 1.f / st.dnorm;
  gm[0] += (gdx - st.dir[0] * rad) * idn;
  gm[1] += (gdy - st.dir[1] * rad) * idn;
  gm[2] += (gdz - st.dir[2] * rad) * idn;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if constexpr (DIRECT) out.d_means[3 * (int64_t)i + k] = gm[k];
    else acc.m[k] += gm[k];
  }
}

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// One thread per Gaussian; MULTI: loop over the views of a batch (records v n + i), else the one view
// `cam0`, passed by value so that its entries are constant-bank operands rather than registers.
// Culled splats (no tile) contribute nothing; a Gaussian culled in every view gets zeros.
// One view: at most 128 registers (4 CTAs per SM). Without the SH staging below, 5 CTAs per SM hid the
// memory latency best (a sweep of 3..8 on GB300: 0.35 / 0.32 / 0.31 / 0.33 / 0.34 / 0.41 ms per 4 calls);
// with it, 4 CTAs per SM take 0.285 ms, while 5 spill and take 0.39.
// The CTAs stride over blocks of 128 Gaussians (a grid of one wave for a single view): while a block
// computes, the next block's lines are already on their way into L2, so that DRAM stays busy through the
// long arithmetic stretch of each block.
template <int DEG, bool VEC, bool MULTI>
__global__ void __launch_bounds__(128, MULTI ? 1 : 4) project_backward_kernel(ngs_gaussians g, const ViewParams* __restrict__ views,
                                                               CamParams cam0, RenderParams rp,
                                                               const uint32_t* tile_count, const float4* grad2d,
                                                               ngs_grads out) {
  pdl_wait();
  constexpr int K = (DEG + 1) * (DEG + 1);
  // One view with 16-byte SH rows: each warp moves its 32 Gaussians' SH blocks (contiguous in memory)
  // between global and shared memory with coalesced 16-byte accesses; each thread then reads its
  // coefficients and writes its SH gradient there (row stride Q + 1 float4 against bank conflicts).
  constexpr bool kStage = VEC && !MULTI;
  constexpr int Q = VEC ? 3 * K / 4 : 1;  // float4 per Gaussian
  __shared__ float4 s_sh[kStage ? 128 * (Q + 1) : 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < g.n; b0 += step) {
    const int i = (int)(b0 + threadIdx.x);
    // every line this Gaussian's chain reads is requested here, together with the warp's SH staging below,
    // so that the loads after the test of its tile count find them in L1 (prefetches hold no registers)
    if (i < g.n) {
      prefetch_l1(g.means + 3 * (int64_t)i);
      prefetch_l1(g.log_scales + 3 * (int64_t)i);
      prefetch_l1(g.quats + 4 * (int64_t)i);
      prefetch_l1(g.opacity_logits + i);
      if constexpr (!MULTI) {
        prefetch_l1(grad2d + 3 * (int64_t)i);
        prefetch_l1(grad2d + 3 * (int64_t)i + 2);
      }
    }
    const int64_t g0 = b0 + warp * 32;  // first Gaussian of the warp
    const int64_t left = g.n - g0;
    const int warp_n = left <= 0 ? 0 : (left >= 32 ? 32 : (int)left);
    float4* my_sh = kStage ? &s_sh[threadIdx.x * (Q + 1)] : nullptr;
    if constexpr (kStage) {
      const float4* src = reinterpret_cast<const float4*>(g.sh) + g0 * Q;
      for (int idx = lane; idx < warp_n * Q; idx += 32) {
        const int j = idx / Q;
        s_sh[(warp * 32 + j) * (Q + 1) + (idx - j * Q)] = src[idx];
      }
      __syncwarp();
    }
    if constexpr (!MULTI) {
      // the next block's lines into L2 (the warp's SH block: Q * 512 bytes, one 128-byte line per lane step)
      const int64_t nx = (int64_t)i + step;
      if (nx < g.n) {
        prefetch_l2(g.means + 3 * nx);
        prefetch_l2(g.log_scales + 3 * nx);
        prefetch_l2(g.quats + 4 * nx);
        prefetch_l2(g.opacity_logits + nx);
        prefetch_l2(grad2d + 3 * nx);
        prefetch_l2(grad2d + 3 * nx + 2);
        prefetch_l2(tile_count + nx);
      }
      if constexpr (kStage) {
        const int64_t ng0 = g0 + step;
        const int64_t nleft = g.n - ng0;
        const int nwarp = nleft <= 0 ? 0 : (nleft >= 32 ? 32 : (int)nleft);
        const char* nsrc = reinterpret_cast<const char*>(reinterpret_cast<const float4*>(g.sh) + ng0 * Q);
        for (int line = lane; line * 128 < nwarp * Q * 16; line += 32) prefetch_l2(nsrc + line * 128);
      }
    }
    if (i < g.n) {
      ParamGrad<DEG> acc;
#pragma unroll
      for (int k = 0; k < 3; ++k) acc.m[k] = acc.ls[k] = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) acc.q[k] = 0.f;
      acc.op = 0.f;
#pragma unroll
      for (int k = 0; k < 3 * K; ++k) acc.sh[k] = 0.f;
      bool written = false;
      if constexpr (!MULTI) {
        if (tile_count[i] != 0) {
          const float* sh_src = kStage ? reinterpret_cast<const float*>(my_sh) : g.sh + (int64_t)i * K * 3;
          float* dsh_dst = kStage ? reinterpret_cast<float*>(my_sh) : out.d_sh + (int64_t)i * K * 3;
          const float4* gr = grad2d + 3 * (int64_t)i;
          add_view_gradient<DEG, VEC, true>(load_params(g, i), cam0, rp, i, gr[0], gr[1], gr[2], acc, out, sh_src,
                                            dsh_dst);
          written = true;
        }
      } else {
        const RawParams prm = load_params(g, i);
        for (int v = 0; v < (int)rp.n_views; ++v) {
          const int64_t r = (int64_t)v * g.n + i;
          if (tile_count[r] == 0) continue;
          const CamParams cam = views[v].cam;
          add_view_gradient<DEG, VEC, false>(prm, cam, rp, i, grad2d[3 * r], grad2d[3 * r + 1], grad2d[3 * r + 2],
                                             acc, out, g.sh + (int64_t)i * K * 3, nullptr);
        }
      }
      if (!written) {  // the sums over views (or zeros: culled in every view)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          out.d_means[3 * (int64_t)i + k] = acc.m[k];
          out.d_log_scales[3 * (int64_t)i + k] = acc.ls[k];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) out.d_quats[4 * (int64_t)i + k] = acc.q[k];
        out.d_opacity_logits[i] = acc.op;
        if constexpr (kStage) store_sh<K, VEC>(reinterpret_cast<float*>(my_sh), acc.sh);
        else store_sh<K, VEC>(out.d_sh + (int64_t)i * K * 3, acc.sh);
      }
    }
    if constexpr (kStage) {
      __syncwarp();
      float4* dst = reinterpret_cast<float4*>(out.d_sh) + g0 * Q;
      for (int idx = lane; idx < warp_n * Q; idx += 32) {
        const int j = idx / Q;
        dst[idx] = s_sh[(warp * 32 + j) * (Q + 1) + (idx - j * Q)];
      }
      __syncwarp();  // the next block's staging overwrites these rows
    }
  }
}

}  // namespace

void launch_project(const ngs_gaussians& g, const ViewParams* views, const CamParams& cam0, const RenderParams& rp,
                    float4* rec, uint32_t* depth_key, uint32_t* tile_count, uint32_t* order, cudaStream_t s) {
  if (g.n == 0) return;
  unsigned blocks = (unsigned)((g.n + 255) / 256) * rp.n_views;
  bool vec = ((uintptr_t)g.sh & 15) == 0;
#define NGS_PROJECT(D, V) \
  launch_pdl(project_kernel<D, V>, blocks, 256, 0, s, g, views, cam0, rp, rec, depth_key, tile_count, order)
  switch (rp.sh_degree) {
    case 0: NGS_PROJECT(0, false); break;
    case 1:
      if (vec) NGS_PROJECT(1, true);
      else NGS_PROJECT(1, false);
      break;
    case 2: NGS_PROJECT(2, false); break;
    default:
      if (vec) NGS_PROJECT(3, true);
      else NGS_PROJECT(3, false);
      break;
  }
#undef NGS_PROJECT
}

void launch_emit_pairs(const float4* rec, const uint32_t* order, const uint32_t* offsets, const ViewParams* views,
                       const RenderParams& rp, uint32_t* tiles, uint32_t* vals, uint32_t cap, cudaStream_t s) {
  if (rp.n_records == 0) return;
  launch_pdl(emit_pairs_kernel, (rp.n_records + 255) / 256, 256, 0, s, rec, order, offsets, views, rp, tiles, vals,
             cap);
}

template <int DEG, bool VEC>
static void project_backward_views(const ngs_gaussians& g, const ViewParams* views, const CamParams& cam0,
                                   const RenderParams& rp, const uint32_t* tile_count, const float4* grad2d,
                                   const ngs_grads& out, int num_sms, cudaStream_t s) {
  const int64_t blocks = (g.n + 127) / 128;
  if (rp.n_views > 1) {
    launch_pdl(project_backward_kernel<DEG, VEC, true>, (unsigned)blocks, 128, 0, s, g, views, cam0, rp, tile_count,
               grad2d, out);
  } else {
    // one wave: 4 CTAs per SM (the kernel's register bound)
    const int64_t wave = 4 * (int64_t)std::max(num_sms, 1);
    launch_pdl(project_backward_kernel<DEG, VEC, false>, (unsigned)std::min(blocks, wave), 128, 0, s, g, views, cam0,
               rp, tile_count, grad2d, out);
  }
}

void launch_project_backward(const ngs_gaussians& g, const ViewParams* views, const CamParams& cam0,
                             const RenderParams& rp, const uint32_t* tile_count, const float4* grad2d,
                             const ngs_grads& out, int num_sms, cudaStream_t s) {
  if (g.n == 0) return;
  bool vec = ((uintptr_t)g.sh & 15) == 0 && ((uintptr_t)out.d_sh & 15) == 0;
  switch (rp.sh_degree) {
    case 0: project_backward_views<0, false>(g, views, cam0, rp, tile_count, grad2d, out, num_sms, s); break;
    case 1:
      if (vec) project_backward_views<1, true>(g, views, cam0, rp, tile_count, grad2d, out, num_sms, s);
      else project_backward_views<1, false>(g, views, cam0, rp, tile_count, grad2d, out, num_sms, s);
      break;
    case 2: project_backward_views<2, false>(g, views, cam0, rp, tile_count, grad2d, out, num_sms, s); break;
    default:
      if (vec) project_backward_views<3, true>(g, views, cam0, rp, tile_count, grad2d, out, num_sms, s);
      else project_backward_views<3, false>(g, views, cam0, rp, tile_count, grad2d, out, num_sms, s);
      break;
  }
}

}  // namespace ngs
