/*
 * ngs_oracle.c -- FP64 CPU oracle for generalized non-exponential Gaussian splatting.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load or run this library. It shares no code, header, table or helper with the CUDA path; the
 * product path never calls it.
 *
 * It computes, plainly and slowly, what the GPU hot path computes:
 *
 *   1. The compositing operator over one depth-ordered list of splats (Sec. 4.2):
 *        L0 = sum_i E_i pbar_i + L_b Tbar_{N+1},  Tbar_i = 1 - sum_{j<i} pbar_j    (Eq. generalized_gaussian)
 *      with pbar_i the slope term of the mother transmittance for i < k, 1 - sum_{j<k} pbar_j at the
 *      saturating splat k, and 0 after it (Eq. nexp_p). Slope terms per model from Table 1:
 *        exponential  alpha_i prod_{j<i}(1 - alpha_j)
 *        quadratic    alpha_i (1 + c taubar_i),  taubar_i = sum_{j<i} alpha_j      (linear: c = 0)
 *        blended      alpha_i (1 - gamma + gamma prod_{j<i}(1 - alpha_j))
 *        Vicini       lerp(pbar^lin, pbar^exp, gamma) of the two already-saturated lists
 *   2. The adjoint of that operator. Quadratic and linear: the paper's recursion of App. C
 *      (Eq. generalized_gaussians_gen, the Theta_i recursion of C.2). Exponential, blended and Vicini:
 *      the paper derives none; the plain derivative of the same sums is written out.
 *   3. Projection of each 3D Gaussian to a screen-space splat: the EWA convention of 3D Gaussian
 *      splatting that Sec. 3 builds on (covariance R S S^T R^T, Jacobian of the pinhole map at the
 *      mean, 2D dilation), opacity aleph = sigmoid(logit), emission E from real spherical harmonics.
 *   4. Per-pixel rendering with no tiles: every splat whose alpha_i(p) = min(alpha_max, aleph_i K_i(p))
 *      reaches alpha_min, ordered front to back by (view depth as FP32, Gaussian index) (Sec. 3, "sorted
 *      front-to-bottom").
 *   5. Gradients w.r.t. the raw parameters: the per-pixel adjoint (2.) chained by hand through alpha_i(p)
 *      to the splat record, then through the projection (3.) by complex-step differentiation, which is
 *      exact to rounding for an analytic map (Squire and Trapp, SIAM Review 1998).
 *
 * Decisions that turn a float into an integer take the GPU kernel's precision where the two can agree
 * exactly: the sort depth is the FP32 value fmaf(r20, x, t2) -> fmaf(r21, y, .) -> fmaf(r22, z, .) and
 * the near-plane test compares that FP32 depth. The remaining threshold decisions (alpha >= alpha_min,
 * the alpha_max clamp, saturation sum >= 1, the exponential T_eps stop) are made in FP64; a pixel where
 * any of them lies within a relative distance `fragile_rel` of its threshold is flagged "fragile" so
 * that parity tests can exclude it.
 *
 * Build: gcc -O2 -std=gnu11 -ffp-contract=off -fPIC -shared ngs_oracle.c -lm -lpthread
 * (-ffp-contract=off keeps results identical on x86-64 and aarch64.)
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EXP 0
#define ORC_QUAD 1
#define ORC_BLEND 2
#define ORC_VICINI 3

#define ORC_REC 10 /* u, v, A, B, C, aleph, E0, E1, E2, rbound */

typedef struct {
  int64_t n;
  int32_t sh_degree;
  const double* means;          /* [n][3] world position */
  const double* log_scales;     /* [n][3] */
  const double* quats;          /* [n][4] (w, x, y, z), any norm > 0 */
  const double* opacity_logits; /* [n] */
  const double* sh;             /* [n][(d+1)^2][3] */
} orc_scene;

typedef struct {
  double viewmat[12]; /* world -> view, row-major [R | t]; the camera looks down +z */
  double fx, fy, cx, cy;
  int32_t width, height;
} orc_camera;

typedef struct {
  int32_t kind; /* ORC_EXP, ORC_QUAD (param = c), ORC_BLEND / ORC_VICINI (param = gamma) */
  double param;
} orc_model;

typedef struct {
  double alpha_min, alpha_max, t_eps, dilation, near_plane;
  double background[3];
  int32_t max_splats; /* 0 = unlimited */
  double fragile_rel;
} orc_opts;

typedef struct {
  int32_t x0, y0, w, h;
} orc_window;

typedef struct {
  double* image;       /* [h][w][3] */
  int32_t* overdraw;   /* [h][w] splats composited, the saturating one included */
  int32_t* n_listed;   /* [h][w] splats with alpha >= alpha_min (may be NULL) */
  uint8_t* fragile;    /* [h][w] (may be NULL) */
  uint64_t* signature; /* [h][w] hash of the composited ids, stop and clamp state (may be NULL) */
} orc_fwd_out;

typedef struct {
  const double* dl_dimage; /* [h][w][3] */
  double* d_means;         /* [n][3] overwritten */
  double* d_log_scales;    /* [n][3] */
  double* d_quats;         /* [n][4] */
  double* d_opacity_logits;/* [n] */
  double* d_sh;            /* [n][(d+1)^2][3] */
  uint8_t* fragile_gauss;  /* [n] a colour channel sits within fragile_rel of the max(0,.) clamp (may be NULL) */
  /* Optional [n]-shaped outputs like the gradients: the sum of the absolute values of every per-pixel term
   * chained through the absolute Jacobian. It is the scale of the rounding error an FP32 accumulation of
   * the same terms can make, whatever their cancellation; tests use it to bound that error. */
  double* s_means;
  double* s_log_scales;
  double* s_quats;
  double* s_opacity_logits;
  double* s_sh;
} orc_bwd;

/* ------------------------------------------------------------------------------------------------
 * 1. Compositing operator over one ordered list (Eq. generalized_gaussian, Eq. nexp_p, Table 1).
 * ------------------------------------------------------------------------------------------------ */

typedef struct {
  int m;            /* list entries composited (overdraw) */
  int saturated;    /* quadratic/blended: the ray saturated at entry m-1 (that entry is k) */
  double color[3];  /* L0, background included */
  double T_end;     /* Tbar after the composited entries */
  double margin;    /* smallest relative distance of a stop decision to its threshold */
  int clamp_fired;  /* the [.]_+ clamp of a quadratic slope term was active */
  int k_lin, k_exp; /* Vicini: entry where its linear list saturated / its exponential list stopped (-1: none) */
} comp_result;

static void margin_update(double* margin, double value, double threshold) {
  double d = fabs(value - threshold) / fabs(threshold);
  if (d < *margin) *margin = d;
}

/* Composite entries 0..n-1 (already filtered by alpha >= alpha_min) front to back. Writes pbar[0..m). */
static void composite(int kind, double param, double t_eps, int max_splats, const double bg[3], int n,
                      const double* alpha, const double* E, double* pbar, comp_result* r) {
  memset(r, 0, sizeof(*r));
  r->margin = INFINITY;
  double C[3] = {0, 0, 0};
  if (kind == ORC_EXP) {
    /* pbar_i = alpha_i T_i with T_i = prod_{j<i}(1 - alpha_j) (Table 1, row 1). The exponential never
     * reaches zero; the ray stops before the splat that would take T below t_eps. */
    double T = 1.0;
    int m = 0;
    for (int i = 0; i < n; ++i) {
      if (max_splats > 0 && m == max_splats) break;
      double testT = T * (1.0 - alpha[i]);
      if (t_eps > 0) {
        margin_update(&r->margin, testT, t_eps);
        if (testT < t_eps) break;
      }
      pbar[i] = alpha[i] * T;
      for (int ch = 0; ch < 3; ++ch) C[ch] += E[3 * i + ch] * pbar[i];
      T = testT;
      ++m;
    }
    r->m = m;
    r->T_end = T;
  } else if (kind == ORC_QUAD || kind == ORC_BLEND) {
    /* pbar_i = slope term while the running sum stays below 1; the splat k whose slope term would reach
     * 1 gets the remainder 1 - sum_{j<k} pbar_j and the ray stops (Eq. nexp_p). */
    double S = 0.0, tau = 0.0, P = 1.0;
    int m = 0;
    for (int i = 0; i < n; ++i) {
      if (max_splats > 0 && m == max_splats) break;
      double pt;
      if (kind == ORC_QUAD) {
        pt = alpha[i] * (1.0 + param * tau);
        if (pt < 0) { pt = 0; r->clamp_fired = 1; }
      } else {
        pt = alpha[i] * (1.0 - param + param * P);
      }
      margin_update(&r->margin, S + pt, 1.0);
      ++m;
      if (S + pt >= 1.0) {
        pbar[i] = 1.0 - S;
        for (int ch = 0; ch < 3; ++ch) C[ch] += E[3 * i + ch] * pbar[i];
        S = 1.0;
        r->saturated = 1;
        break;
      }
      pbar[i] = pt;
      for (int ch = 0; ch < 3; ++ch) C[ch] += E[3 * i + ch] * pt;
      S += pt;
      tau += alpha[i];
      P *= 1.0 - alpha[i];
    }
    r->m = m;
    r->T_end = r->saturated ? 0.0 : 1.0 - S;
  } else { /* ORC_VICINI: lerp of the saturated linear list and the exponential list */
    double gam = param, Sl = 0.0, Te = 1.0;
    int sat_l = 0, stop_e = 0, m = 0;
    r->k_lin = r->k_exp = -1;
    for (int i = 0; i < n; ++i) {
      if (max_splats > 0 && m == max_splats) break;
      double pe = 0.0, pl = 0.0;
      if (!stop_e) {
        double testT = Te * (1.0 - alpha[i]);
        if (t_eps > 0) {
          margin_update(&r->margin, testT, t_eps);
          if (testT < t_eps) { stop_e = 1; r->k_exp = i; }
        }
        if (!stop_e) { pe = alpha[i] * Te; Te = testT; }
      }
      if (sat_l && stop_e) break;
      if (!sat_l) {
        margin_update(&r->margin, Sl + alpha[i], 1.0);
        if (Sl + alpha[i] >= 1.0) { pl = 1.0 - Sl; Sl = 1.0; sat_l = 1; r->k_lin = i; }
        else { pl = alpha[i]; Sl += alpha[i]; }
      }
      pbar[i] = (1.0 - gam) * pl + gam * pe;
      for (int ch = 0; ch < 3; ++ch) C[ch] += E[3 * i + ch] * pbar[i];
      ++m;
    }
    r->m = m;
    r->T_end = (1.0 - gam) * (1.0 - Sl) + gam * Te;
  }
  for (int ch = 0; ch < 3; ++ch) r->color[ch] = C[ch] + bg[ch] * r->T_end;
}

/* Adjoint of composite(): given g = dL/dL0 (RGB), write dL/dalpha_i and dL/dE_i for i < m. */
static void composite_adjoint(int kind, double param, double t_eps, const double bg[3], const comp_result* r,
                              const double* alpha, const double* E, const double* pbar, const double g[3],
                              double* dalpha, double* dE) {
  int m = r->m;
  for (int i = 0; i < m; ++i) {
    dalpha[i] = 0;
    for (int ch = 0; ch < 3; ++ch) dE[3 * i + ch] = g[ch] * pbar[i];
  }
  if (m == 0) return;
  if (kind == ORC_QUAD) {
    /* App. C: L0 = sum_{i<k} DeltaE_i pbar_i + E_k with DeltaE_i = E_i - E_k; E_k = L_b when the ray
     * never saturates (k = N+1). For i < k:
     *   dL0/dalpha_i = DeltaE_i (1 + c taubar_i) + c Theta_i,   Theta_0 = sum_{j=1}^{k-1} DeltaE_j alpha_j,
     *   Theta_i = Theta_{i-1} - DeltaE_i alpha_i;   dL0/dalpha_k = 0;   dL0/dE_i = pbar_i (i <= k). */
    double c = param;
    int k = r->saturated ? m - 1 : m;
    const double* Ek = r->saturated ? &E[3 * k] : bg;
    double Theta[3] = {0, 0, 0};
    for (int j = 1; j < k; ++j)
      for (int ch = 0; ch < 3; ++ch) Theta[ch] += (E[3 * j + ch] - Ek[ch]) * alpha[j];
    double tau = 0;
    for (int i = 0; i < k; ++i) {
      if (i > 0)
        for (int ch = 0; ch < 3; ++ch) Theta[ch] -= (E[3 * i + ch] - Ek[ch]) * alpha[i];
      double s = 0;
      for (int ch = 0; ch < 3; ++ch) s += g[ch] * ((E[3 * i + ch] - Ek[ch]) * (1.0 + c * tau) + c * Theta[ch]);
      dalpha[i] = s;
      tau += alpha[i];
    }
  } else if (kind == ORC_EXP) {
    /* L0 = sum_i E_i alpha_i T_i + L_b T_m. With U_i the radiance arriving at splat i from behind it,
     * U_{m-1} = L_b and U_{i-1} = E_i alpha_i + (1 - alpha_i) U_i (the recursive over operator of
     * App. B), dL0/dalpha_i = T_i (E_i - U_i). */
    double* U = (double*)malloc(sizeof(double) * 3 * m);
    for (int ch = 0; ch < 3; ++ch) U[3 * (m - 1) + ch] = bg[ch];
    for (int i = m - 1; i > 0; --i)
      for (int ch = 0; ch < 3; ++ch)
        U[3 * (i - 1) + ch] = E[3 * i + ch] * alpha[i] + (1.0 - alpha[i]) * U[3 * i + ch];
    double T = 1.0;
    for (int i = 0; i < m; ++i) {
      double s = 0;
      for (int ch = 0; ch < 3; ++ch) s += g[ch] * T * (E[3 * i + ch] - U[3 * i + ch]);
      dalpha[i] = s;
      T *= 1.0 - alpha[i];
    }
    free(U);
  } else if (kind == ORC_BLEND) {
    /* L0 = sum_{i<k} DeltaE_i alpha_i (1 - gamma + gamma P_i) + E_k, P_i = prod_{j<i}(1 - alpha_j).
     * dL0/dalpha_i = DeltaE_i (1 - gamma + gamma P_i) - gamma P_i W_i with
     * W_i = sum_{i<l<k} DeltaE_l alpha_l prod_{i<j<l}(1 - alpha_j), W_{k-1} = 0,
     * W_{i-1} = DeltaE_i alpha_i + (1 - alpha_i) W_i. */
    double gam = param;
    int k = r->saturated ? m - 1 : m;
    const double* Ek = r->saturated ? &E[3 * k] : bg;
    if (k > 0) {
      double* W = (double*)malloc(sizeof(double) * 3 * k);
      for (int ch = 0; ch < 3; ++ch) W[3 * (k - 1) + ch] = 0;
      for (int i = k - 1; i > 0; --i)
        for (int ch = 0; ch < 3; ++ch)
          W[3 * (i - 1) + ch] = (E[3 * i + ch] - Ek[ch]) * alpha[i] + (1.0 - alpha[i]) * W[3 * i + ch];
      double P = 1.0;
      for (int i = 0; i < k; ++i) {
        double s = 0;
        for (int ch = 0; ch < 3; ++ch)
          s += g[ch] * ((E[3 * i + ch] - Ek[ch]) * (1.0 - gam + gam * P) - gam * P * W[3 * i + ch]);
        dalpha[i] = s;
        P *= 1.0 - alpha[i];
      }
      free(W);
    }
  } else { /* ORC_VICINI: (1 - gamma) x linear adjoint + gamma x exponential adjoint over each list */
    double gam = param;
    double* p2 = (double*)malloc(sizeof(double) * (size_t)m);
    double* d2 = (double*)malloc(sizeof(double) * (size_t)m);
    double* dE2 = (double*)malloc(sizeof(double) * 3 * (size_t)m);
    comp_result rl, re;
    /* linear part: its own saturating list over the same entries (no t_eps stop) */
    composite(ORC_QUAD, 0.0, 0.0, 0, bg, m, alpha, E, p2, &rl);
    composite_adjoint(ORC_QUAD, 0.0, 0.0, bg, &rl, alpha, E, p2, g, d2, dE2);
    for (int i = 0; i < rl.m; ++i) dalpha[i] += (1.0 - gam) * d2[i];
    /* exponential part, with its own T_eps stop */
    composite(ORC_EXP, 0.0, t_eps, 0, bg, m, alpha, E, p2, &re);
    composite_adjoint(ORC_EXP, 0.0, t_eps, bg, &re, alpha, E, p2, g, d2, dE2);
    for (int i = 0; i < re.m; ++i) dalpha[i] += gam * d2[i];
    free(p2);
    free(d2);
    free(dE2);
  }
}

/* ------------------------------------------------------------------------------------------------
 * 3. Projection (EWA splatting convention of Sec. 3's 3DGS baseline), in complex arithmetic so that a
 *    complex step on any input yields the exact derivative of every output.
 * ------------------------------------------------------------------------------------------------ */

typedef double complex cplx;

/* Real spherical harmonics up to degree 3 at unit direction (x, y, z), in the coefficient order and
 * sign convention of 3D Gaussian splatting assets (Condon-Shortley phase). Normalisations are the
 * closed forms sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times sqrt(2) for m != 0. */
static int sh_basis(int degree, cplx x, cplx y, cplx z, cplx* Y) {
  const double pi = 3.14159265358979323846;
  int n = 0;
  Y[n++] = 0.5 * sqrt(1.0 / pi);
  if (degree < 1) return n;
  double c1 = sqrt(3.0 / (4.0 * pi));
  Y[n++] = -c1 * y;
  Y[n++] = c1 * z;
  Y[n++] = -c1 * x;
  if (degree < 2) return n;
  double c2a = sqrt(15.0 / (4.0 * pi)), c2b = sqrt(5.0 / (16.0 * pi)), c2c = sqrt(15.0 / (16.0 * pi));
  Y[n++] = c2a * x * y;
  Y[n++] = -c2a * y * z;
  Y[n++] = c2b * (2.0 * z * z - x * x - y * y);
  Y[n++] = -c2a * x * z;
  Y[n++] = c2c * (x * x - y * y);
  if (degree < 3) return n;
  double c3a = sqrt(35.0 / (32.0 * pi)), c3b = sqrt(105.0 / (4.0 * pi)), c3c = sqrt(21.0 / (32.0 * pi));
  double c3d = sqrt(7.0 / (16.0 * pi)), c3e = sqrt(105.0 / (16.0 * pi));
  Y[n++] = -c3a * y * (3.0 * x * x - y * y);
  Y[n++] = c3b * x * y * z;
  Y[n++] = -c3c * y * (4.0 * z * z - x * x - y * y);
  Y[n++] = c3d * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
  Y[n++] = -c3c * x * (4.0 * z * z - x * x - y * y);
  Y[n++] = c3e * z * (x * x - y * y);
  Y[n++] = -c3a * x * (x * x - 3.0 * y * y);
  return n;
}

/* Inputs in complex form: p[3], s[3], q[4], logit, sh[K*3]. Output rec[9] = u, v, A, B, C, aleph, E0..2,
 * plus (real only) the 2D covariance's largest eigenvalue. Returns 0 when the splat cannot be formed. */
static int project_c(const orc_camera* cam, double dilation, int K, const cplx* p, const cplx* s,
                     const cplx* q, cplx logit, const cplx* sh, cplx* rec, double* lam_max, double* e_real) {
  const double* V = cam->viewmat;
  cplx pv[3];
  for (int r = 0; r < 3; ++r) pv[r] = V[4 * r + 0] * p[0] + V[4 * r + 1] * p[1] + V[4 * r + 2] * p[2] + V[4 * r + 3];
  cplx x = pv[0], y = pv[1], z = pv[2];
  /* pinhole map: u = fx x / z + cx, v = fy y / z + cy */
  rec[0] = cam->fx * x / z + cam->cx;
  rec[1] = cam->fy * y / z + cam->cy;
  /* rotation from the normalised quaternion (w, x, y, z) */
  cplx nq = csqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  cplx w = q[0] / nq, a = q[1] / nq, b = q[2] / nq, c = q[3] / nq;
  cplx Rq[3][3] = {
      {1.0 - 2.0 * (b * b + c * c), 2.0 * (a * b - w * c), 2.0 * (a * c + w * b)},
      {2.0 * (a * b + w * c), 1.0 - 2.0 * (a * a + c * c), 2.0 * (b * c - w * a)},
      {2.0 * (a * c - w * b), 2.0 * (b * c + w * a), 1.0 - 2.0 * (a * a + b * b)},
  };
  /* world covariance Sigma = Rq S S^T Rq^T, S = diag(exp(s)) */
  cplx M[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[i][j] = Rq[i][j] * cexp(s[j]);
  cplx Sig[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Sig[i][j] = M[i][0] * M[j][0] + M[i][1] * M[j][1] + M[i][2] * M[j][2];
  /* T = J W with J the Jacobian of the pinhole map at the mean, W the view rotation */
  cplx J[2][3] = {{cam->fx / z, 0.0, -cam->fx * x / (z * z)}, {0.0, cam->fy / z, -cam->fy * y / (z * z)}};
  cplx T[2][3];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) T[i][j] = J[i][0] * V[0 + j] + J[i][1] * V[4 + j] + J[i][2] * V[8 + j];
  /* 2D covariance T Sigma T^T + dilation I */
  cplx TS[2][3];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) TS[i][j] = T[i][0] * Sig[0][j] + T[i][1] * Sig[1][j] + T[i][2] * Sig[2][j];
  cplx s00 = TS[0][0] * T[0][0] + TS[0][1] * T[0][1] + TS[0][2] * T[0][2] + dilation;
  cplx s01 = TS[0][0] * T[1][0] + TS[0][1] * T[1][1] + TS[0][2] * T[1][2];
  cplx s11 = TS[1][0] * T[1][0] + TS[1][1] * T[1][1] + TS[1][2] * T[1][2] + dilation;
  cplx det = s00 * s11 - s01 * s01;
  if (!(creal(det) > 0)) return 0;
  rec[2] = s11 / det;  /* conic A */
  rec[3] = -s01 / det; /* conic B */
  rec[4] = s00 / det;  /* conic C */
  double ha = 0.5 * (creal(s00) + creal(s11)), hd = 0.5 * (creal(s00) - creal(s11));
  *lam_max = ha + sqrt(hd * hd + creal(s01) * creal(s01));
  rec[5] = 1.0 / (1.0 + cexp(-logit));
  /* emission: E = max(0, 1/2 + sum_lm Y_lm(d) sh_lm), d the unit direction from the camera centre */
  double cc[3];
  for (int j = 0; j < 3; ++j) cc[j] = -(V[0 + j] * V[3] + V[4 + j] * V[7] + V[8 + j] * V[11]);
  cplx d0 = p[0] - cc[0], d1 = p[1] - cc[1], d2 = p[2] - cc[2];
  cplx dn = csqrt(d0 * d0 + d1 * d1 + d2 * d2);
  cplx Y[16];
  int deg = 0;
  while ((deg + 1) * (deg + 1) < K) ++deg;
  sh_basis(deg, d0 / dn, d1 / dn, d2 / dn, Y);
  for (int ch = 0; ch < 3; ++ch) {
    cplx e = 0.5;
    for (int k = 0; k < K; ++k) e += Y[k] * sh[3 * k + ch];
    e_real[ch] = creal(e);
    rec[6 + ch] = creal(e) < 0 ? 0.0 : e;
  }
  return 1;
}

/* FP32 depth of the mean, the value both sides sort by: fma chain r20 x -> r21 y -> r22 z onto t2. */
static float depth32(const orc_camera* cam, const double* p) {
  const double* V = cam->viewmat;
  float z = fmaf((float)V[8], (float)p[0], (float)V[11]);
  z = fmaf((float)V[9], (float)p[1], z);
  z = fmaf((float)V[10], (float)p[2], z);
  return z;
}

typedef struct {
  double rec[ORC_REC];
  double e_real[3];
  float z32;
  int valid;
} splat_d;

static int sh_count(int degree) { return (degree + 1) * (degree + 1); }

static void project_one(const orc_scene* sc, const orc_camera* cam, const orc_opts* o, int64_t g, splat_d* out) {
  int K = sh_count(sc->sh_degree);
  cplx p[3], s[3], q[4], sh[48], rec[9];
  for (int j = 0; j < 3; ++j) { p[j] = sc->means[3 * g + j]; s[j] = sc->log_scales[3 * g + j]; }
  for (int j = 0; j < 4; ++j) q[j] = sc->quats[4 * g + j];
  for (int j = 0; j < 3 * K; ++j) sh[j] = sc->sh[(int64_t)3 * K * g + j];
  memset(out, 0, sizeof(*out));
  out->z32 = depth32(cam, &sc->means[3 * g]);
  /* near plane on the FP32 depth */
  if (!(out->z32 > (float)o->near_plane)) return;
  double lam = 0;
  if (!project_c(cam, o->dilation, K, p, s, q, sc->opacity_logits[g], sh, rec, &lam, out->e_real)) return;
  for (int j = 0; j < 9; ++j) out->rec[j] = creal(rec[j]);
  double aleph = out->rec[5];
  if (!(aleph >= o->alpha_min)) return; /* alpha = aleph K <= aleph never reaches alpha_min */
  /* alpha >= alpha_min  <=>  d^T Sigma'^{-1} d <= 2 ln(aleph / alpha_min)  =>  |d|^2 <= 2 ln(.) lam_max */
  out->rec[9] = sqrt(2.0 * log(aleph / o->alpha_min) * lam);
  out->valid = 1;
}

/* ------------------------------------------------------------------------------------------------
 * 4./5. Per-pixel rendering and its adjoint.
 * ------------------------------------------------------------------------------------------------ */

typedef struct {
  float z32;
  int32_t g;    /* local splat index */
  double alpha;
  int clamped;  /* alpha_max clamp active */
} entry;

static int entry_cmp(const void* a, const void* b) {
  const entry* x = (const entry*)a;
  const entry* y = (const entry*)b;
  if (x->z32 < y->z32) return -1;
  if (x->z32 > y->z32) return 1;
  return (x->g > y->g) - (x->g < y->g);
}

typedef struct {
  const orc_scene* sc;
  const orc_camera* cam;
  const orc_model* model;
  const orc_opts* o;
  const orc_window* win;
  const splat_d* sp;     /* local splats */
  const int64_t* gid;    /* local -> global index */
  int64_t nloc;
  const int64_t* start;  /* per pixel offsets into ent */
  entry* ent;
  uint8_t* px_fragile;
  orc_fwd_out* fwd;
  orc_bwd* bwd;
  double* grad_rec;      /* per thread [nthreads][nloc][9] */
  int nthreads;
} render_job;

typedef struct {
  render_job* job;
  int tid;
} worker_arg;

static uint64_t fnv(uint64_t h, uint64_t v) {
  for (int i = 0; i < 8; ++i) { h ^= (v >> (8 * i)) & 0xff; h *= 1099511628211ULL; }
  return h;
}

static void* render_rows(void* argp) {
  worker_arg* wa = (worker_arg*)argp;
  render_job* J = wa->job;
  const orc_window* w = J->win;
  int kind = J->model->kind;
  double par = J->model->param;
  double* grec = J->grad_rec ? J->grad_rec + (size_t)wa->tid * (size_t)J->nloc * 18 : NULL;
  int cap = 0;
  double *alpha = NULL, *E = NULL, *pbar = NULL, *dal = NULL, *dE = NULL;
  for (int yy = wa->tid; yy < w->h; yy += J->nthreads) {
    for (int xx = 0; xx < w->w; ++xx) {
      int64_t pix = (int64_t)yy * w->w + xx;
      entry* L = J->ent + J->start[pix];
      int n = (int)(J->start[pix + 1] - J->start[pix]);
      qsort(L, (size_t)n, sizeof(entry), entry_cmp);
      if (n > cap) {
        cap = n;
        alpha = (double*)realloc(alpha, sizeof(double) * cap);
        E = (double*)realloc(E, sizeof(double) * 3 * cap);
        pbar = (double*)realloc(pbar, sizeof(double) * cap);
        dal = (double*)realloc(dal, sizeof(double) * cap);
        dE = (double*)realloc(dE, sizeof(double) * 3 * cap);
      }
      for (int i = 0; i < n; ++i) {
        alpha[i] = L[i].alpha;
        for (int ch = 0; ch < 3; ++ch) E[3 * i + ch] = J->sp[L[i].g].rec[6 + ch];
      }
      comp_result r;
      composite(kind, par, J->o->t_eps, J->o->max_splats, J->o->background, n, alpha, E, pbar, &r);
      for (int ch = 0; ch < 3; ++ch) J->fwd->image[3 * pix + ch] = r.color[ch];
      J->fwd->overdraw[pix] = r.m;
      if (J->fwd->n_listed) J->fwd->n_listed[pix] = n;
      int fr = J->px_fragile[pix] || r.margin < J->o->fragile_rel || r.clamp_fired;
      for (int i = 0; i < r.m; ++i)
        if (L[i].clamped == 2) fr = 1; /* within fragile_rel of the alpha_max clamp */
      if (J->fwd->fragile) J->fwd->fragile[pix] = (uint8_t)fr;
      if (J->fwd->signature) {
        uint64_t h = 1469598103934665603ULL;
        for (int i = 0; i < r.m; ++i) h = fnv(h, (uint64_t)J->gid[L[i].g] * 4 + (uint64_t)(L[i].clamped == 1));
        h = fnv(h, (uint64_t)r.m * 2 + (uint64_t)r.saturated);
        if (kind == ORC_VICINI) h = fnv(h, ((uint64_t)(r.k_lin + 1) << 32) | (uint64_t)(r.k_exp + 1));
        J->fwd->signature[pix] = h;
      }
      if (grec) {
        const double* g = &J->bwd->dl_dimage[3 * pix];
        if (g[0] == 0 && g[1] == 0 && g[2] == 0) continue;
        composite_adjoint(kind, par, J->o->t_eps, J->o->background, &r, alpha, E, pbar, g, dal, dE);
        double px = J->win->x0 + xx + 0.5, py = J->win->y0 + yy + 0.5;
        for (int i = 0; i < r.m; ++i) {
          const splat_d* s = &J->sp[L[i].g];
          double* gr = grec + (size_t)L[i].g * 18;
          double* ga = gr + 9; /* absolute values of the same terms */
          for (int ch = 0; ch < 3; ++ch) {
            gr[6 + ch] += dE[3 * i + ch];
            ga[6 + ch] += fabs(dE[3 * i + ch]);
          }
          if (L[i].clamped == 1) continue; /* alpha = alpha_max does not depend on the splat */
          /* alpha = aleph exp(-q/2), q = A dx^2 + 2 B dx dy + C dy^2, (dx, dy) = p - (u, v) */
          double dx = px - s->rec[0], dy = py - s->rec[1];
          double A = s->rec[2], B = s->rec[3], C = s->rec[4];
          double q = A * dx * dx + 2.0 * B * dx * dy + C * dy * dy;
          double G = exp(-0.5 * q);
          double a = L[i].alpha;
          double dq = dal[i] * (-0.5 * a);
          double t[6] = {dq * (-2.0 * (A * dx + B * dy)), dq * (-2.0 * (B * dx + C * dy)), dq * dx * dx,
                         dq * 2.0 * dx * dy, dq * dy * dy, dal[i] * G};
          for (int r = 0; r < 6; ++r) {
            gr[r] += t[r];
            ga[r] += fabs(t[r]);
          }
        }
      }
    }
  }
  free(alpha); free(E); free(pbar); free(dal); free(dE);
  return NULL;
}

/* Complex-step chain from record gradients to raw-parameter gradients for one Gaussian. */
static void chain_to_params(const orc_scene* sc, const orc_camera* cam, const orc_opts* o, int64_t g,
                            const double* grec, const double* gabs, orc_bwd* b) {
  int K = sh_count(sc->sh_degree);
  int np = 3 + 3 + 4 + 1 + 3 * K;
  double h = 1e-30;
  for (int j = 0; j < np; ++j) {
    cplx p[3], s[3], q[4], sh[48], rec[9], logit;
    double lam, er[3];
    for (int t = 0; t < 3; ++t) { p[t] = sc->means[3 * g + t]; s[t] = sc->log_scales[3 * g + t]; }
    for (int t = 0; t < 4; ++t) q[t] = sc->quats[4 * g + t];
    for (int t = 0; t < 3 * K; ++t) sh[t] = sc->sh[(int64_t)3 * K * g + t];
    logit = sc->opacity_logits[g];
    double* dst;
    double* sdst;
    if (j < 3) { p[j] += I * h; dst = &b->d_means[3 * g + j]; sdst = b->s_means ? &b->s_means[3 * g + j] : NULL; }
    else if (j < 6) {
      s[j - 3] += I * h;
      dst = &b->d_log_scales[3 * g + j - 3];
      sdst = b->s_log_scales ? &b->s_log_scales[3 * g + j - 3] : NULL;
    } else if (j < 10) {
      q[j - 6] += I * h;
      dst = &b->d_quats[4 * g + j - 6];
      sdst = b->s_quats ? &b->s_quats[4 * g + j - 6] : NULL;
    } else if (j == 10) {
      logit += I * h;
      dst = &b->d_opacity_logits[g];
      sdst = b->s_opacity_logits ? &b->s_opacity_logits[g] : NULL;
    } else {
      sh[j - 11] += I * h;
      dst = &b->d_sh[(int64_t)3 * K * g + j - 11];
      sdst = b->s_sh ? &b->s_sh[(int64_t)3 * K * g + j - 11] : NULL;
    }
    if (!project_c(cam, o->dilation, K, p, s, q, logit, sh, rec, &lam, er)) continue;
    double acc = 0, sacc = 0;
    for (int r = 0; r < 9; ++r) {
      acc += grec[r] * cimag(rec[r]) / h;
      if (gabs) sacc += gabs[r] * fabs(cimag(rec[r]) / h);
    }
    *dst = acc;
    if (sdst) *sdst = sacc;
  }
}

int orc_project(const orc_scene* sc, const orc_camera* cam, const orc_opts* o, double* rec, float* z32,
                int32_t* valid) {
  for (int64_t g = 0; g < sc->n; ++g) {
    splat_d s;
    project_one(sc, cam, o, g, &s);
    memcpy(&rec[ORC_REC * g], s.rec, sizeof(s.rec));
    z32[g] = s.z32;
    valid[g] = s.valid;
  }
  return 0;
}

/* Jacobian of the record (u, v, A, B, C, aleph, E0, E1, E2) w.r.t. the raw parameters of Gaussian g,
 * [9][np] with np = 11 + 3 K, by complex step. */
int orc_project_jacobian(const orc_scene* sc, const orc_camera* cam, const orc_opts* o, int64_t g, double* jac) {
  int K = sh_count(sc->sh_degree);
  int np = 11 + 3 * K;
  orc_bwd b;
  /* chain_to_params with a unit record gradient, one record entry at a time */
  double* dm = (double*)calloc((size_t)sc->n * 3, sizeof(double));
  double* ds = (double*)calloc((size_t)sc->n * 3, sizeof(double));
  double* dq = (double*)calloc((size_t)sc->n * 4, sizeof(double));
  double* dl = (double*)calloc((size_t)sc->n, sizeof(double));
  double* dh = (double*)calloc((size_t)sc->n * 3 * K, sizeof(double));
  memset(&b, 0, sizeof(b));
  b.d_means = dm; b.d_log_scales = ds; b.d_quats = dq; b.d_opacity_logits = dl; b.d_sh = dh;
  for (int r = 0; r < 9; ++r) {
    double e[9] = {0};
    e[r] = 1.0;
    chain_to_params(sc, cam, o, g, e, NULL, &b);
    double* row = jac + (size_t)r * np;
    for (int t = 0; t < 3; ++t) row[t] = dm[3 * g + t];
    for (int t = 0; t < 3; ++t) row[3 + t] = ds[3 * g + t];
    for (int t = 0; t < 4; ++t) row[6 + t] = dq[4 * g + t];
    row[10] = dl[g];
    for (int t = 0; t < 3 * K; ++t) row[11 + t] = dh[(int64_t)3 * K * g + t];
  }
  free(dm); free(ds); free(dq); free(dl); free(dh);
  return 0;
}

/* Render a window of the camera's image. brute_force = 1 tests every valid splat at every pixel;
 * otherwise a splat is only tested at pixels whose centre lies in the bounding box of its disc
 * |d| <= rbound, outside of which alpha < alpha_min holds by the eigenvalue bound (project_one). */
int orc_render(const orc_scene* sc, const orc_camera* cam, const orc_model* model, const orc_opts* o,
               const orc_window* win, int nthreads, int brute_force, orc_fwd_out* fwd, orc_bwd* bwd) {
  if (nthreads < 1) nthreads = 1;
  int64_t n = sc->n;
  int64_t npx = (int64_t)win->w * win->h;
  /* project, keep the splats that can reach the window */
  splat_d* all = (splat_d*)malloc(sizeof(splat_d) * (size_t)(n > 0 ? n : 1));
  int64_t* gid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t nloc = 0;
  for (int64_t g = 0; g < n; ++g) {
    splat_d s;
    project_one(sc, cam, o, g, &s);
    if (!s.valid) continue;
    if (!brute_force) {
      double rb = s.rec[9] + 1e-6;
      if (s.rec[0] + rb < win->x0 || s.rec[0] - rb > win->x0 + win->w) continue;
      if (s.rec[1] + rb < win->y0 || s.rec[1] - rb > win->y0 + win->h) continue;
    }
    all[nloc] = s;
    gid[nloc] = g;
    ++nloc;
  }
  /* gather: two passes (count, fill) over (splat, pixel) pairs */
  int64_t* start = (int64_t*)calloc((size_t)npx + 1, sizeof(int64_t));
  uint8_t* pxf = (uint8_t*)calloc((size_t)npx + 1, 1);
  entry* ent = NULL;
  for (int pass = 0; pass < 2; ++pass) {
    int64_t* cursor = NULL;
    if (pass == 1) {
      for (int64_t p = 0; p < npx; ++p) start[p + 1] += start[p];
      ent = (entry*)malloc(sizeof(entry) * (size_t)(start[npx] > 0 ? start[npx] : 1));
      cursor = (int64_t*)malloc(sizeof(int64_t) * (size_t)(npx > 0 ? npx : 1));
      memcpy(cursor, start, sizeof(int64_t) * (size_t)npx);
    }
    for (int64_t l = 0; l < nloc; ++l) {
      const splat_d* s = &all[l];
      int x0 = 0, x1 = win->w - 1, y0 = 0, y1 = win->h - 1;
      if (!brute_force) {
        double rb = s->rec[9] + 1e-6;
        x0 = (int)fmax(0.0, ceil(s->rec[0] - rb - 0.5) - win->x0);
        x1 = (int)fmin((double)win->w - 1, floor(s->rec[0] + rb - 0.5) - win->x0);
        y0 = (int)fmax(0.0, ceil(s->rec[1] - rb - 0.5) - win->y0);
        y1 = (int)fmin((double)win->h - 1, floor(s->rec[1] + rb - 0.5) - win->y0);
      }
      for (int yy = y0; yy <= y1; ++yy) {
        for (int xx = x0; xx <= x1; ++xx) {
          double px = win->x0 + xx + 0.5, py = win->y0 + yy + 0.5;
          double dx = px - s->rec[0], dy = py - s->rec[1];
          double q = s->rec[2] * dx * dx + 2.0 * s->rec[3] * dx * dy + s->rec[4] * dy * dy;
          double raw = s->rec[5] * exp(-0.5 * q);
          double a = raw < o->alpha_max ? raw : o->alpha_max;
          int64_t pix = (int64_t)yy * win->w + xx;
          if (pass == 0) {
            if (fabs(a - o->alpha_min) < o->fragile_rel * o->alpha_min) pxf[pix] = 1;
            if (a >= o->alpha_min) start[pix + 1]++;
          } else if (a >= o->alpha_min) {
            entry* e = &ent[cursor[pix]++];
            e->z32 = s->z32;
            e->g = (int32_t)l;
            e->alpha = a;
            e->clamped = raw >= o->alpha_max ? 1 : 0;
            if (fabs(raw - o->alpha_max) < o->fragile_rel * o->alpha_max) e->clamped = e->clamped ? 1 : 2;
            if (fabs(raw - o->alpha_max) < o->fragile_rel * o->alpha_max) pxf[pix] = 1;
          }
        }
      }
    }
    free(cursor);
  }
  render_job job;
  memset(&job, 0, sizeof(job));
  job.sc = sc; job.cam = cam; job.model = model; job.o = o; job.win = win;
  job.sp = all; job.gid = gid; job.nloc = nloc; job.start = start; job.ent = ent;
  job.px_fragile = pxf; job.fwd = fwd; job.bwd = bwd; job.nthreads = nthreads;
  if (bwd) job.grad_rec = (double*)calloc((size_t)nthreads * (size_t)nloc * 18 + 1, sizeof(double));
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
  worker_arg* wa = (worker_arg*)malloc(sizeof(worker_arg) * nthreads);
  for (int t = 0; t < nthreads; ++t) {
    wa[t].job = &job;
    wa[t].tid = t;
    if (t > 0) pthread_create(&th[t], NULL, render_rows, &wa[t]);
  }
  render_rows(&wa[0]);
  for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
  if (bwd) {
    int K = sh_count(sc->sh_degree);
    memset(bwd->d_means, 0, sizeof(double) * 3 * (size_t)n);
    memset(bwd->d_log_scales, 0, sizeof(double) * 3 * (size_t)n);
    memset(bwd->d_quats, 0, sizeof(double) * 4 * (size_t)n);
    memset(bwd->d_opacity_logits, 0, sizeof(double) * (size_t)n);
    memset(bwd->d_sh, 0, sizeof(double) * 3 * (size_t)K * (size_t)n);
    if (bwd->fragile_gauss) memset(bwd->fragile_gauss, 0, (size_t)n);
    double* sarr[5] = {bwd->s_means, bwd->s_log_scales, bwd->s_quats, bwd->s_opacity_logits, bwd->s_sh};
    size_t swid[5] = {3, 3, 4, 1, 3 * (size_t)K};
    for (int k = 0; k < 5; ++k)
      if (sarr[k]) memset(sarr[k], 0, sizeof(double) * swid[k] * (size_t)n);
    for (int64_t l = 0; l < nloc; ++l) {
      double gr[18] = {0};
      for (int t = 0; t < nthreads; ++t)
        for (int r = 0; r < 18; ++r) gr[r] += job.grad_rec[((size_t)t * nloc + l) * 18 + r];
      int nz = 0;
      for (int r = 0; r < 18; ++r) nz |= gr[r] != 0;
      if (!nz) continue;
      chain_to_params(sc, cam, o, gid[l], gr, gr + 9, bwd);
      if (bwd->fragile_gauss)
        for (int ch = 0; ch < 3; ++ch)
          if (fabs(all[l].e_real[ch]) < o->fragile_rel) bwd->fragile_gauss[gid[l]] = 1;
    }
    free(job.grad_rec);
  }
  free(th); free(wa); free(all); free(gid); free(start); free(pxf); free(ent);
  return 0;
}

/* The compositing operator alone over one list (no geometry, no alpha_min filter): pbar[0..n) (zeros past
 * the stop), and out4 = {color r, g, b, T_end}; returns m. With g != NULL also writes the adjoint. */
int orc_composite_list(int32_t kind, double param, double t_eps, int32_t max_splats, const double* bg, int32_t n,
                       const double* alpha, const double* E, double* pbar, double* out4, int32_t* saturated,
                       const double* g, double* dalpha, double* dE) {
  for (int i = 0; i < n; ++i) pbar[i] = 0;
  comp_result r;
  composite(kind, param, t_eps, max_splats, bg, n, alpha, E, pbar, &r);
  for (int ch = 0; ch < 3; ++ch) out4[ch] = r.color[ch];
  out4[3] = r.T_end;
  if (saturated) *saturated = r.saturated;
  if (g) {
    for (int i = 0; i < n; ++i) { dalpha[i] = 0; dE[3 * i] = dE[3 * i + 1] = dE[3 * i + 2] = 0; }
    composite_adjoint(kind, param, t_eps, bg, &r, alpha, E, pbar, g, dalpha, dE);
  }
  return r.m;
}
