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
 * the alpha_max clamp, saturation sum >= 1, the exponential T_eps stop, the max(0, .) of a colour channel)
 * are made in FP64. Where such a value lies within a stated first-order bound of the error the GPU's FP32
 * computation of it can make (alpha_band(), composite(), project_c()), the decision is "borderline": both
 * ways are legitimate results of the method in FP32. The oracle then enumerates every combination of the
 * borderline decisions of a pixel's walk and reports each outcome (orc_alt_out), so that a test can check
 * that the GPU's pixel is one of them rather than leave the pixel out.

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
} orc_opts;

typedef struct {
  int32_t x0, y0, w, h;
} orc_window;

typedef struct {
  double* image;       /* [h][w][3] */
  int32_t* overdraw;   /* [h][w] splats composited, the saturating one included */
  int32_t* n_listed;   /* [h][w] splats with alpha >= alpha_min (may be NULL) */
  uint8_t* fragile;    /* [h][w] 0: no borderline decision; 1: several outcomes (all enumerated when an
                          orc_alt_out is given); 2: unresolved (more than ORC_MAX_OUTCOMES outcomes, a
                          bound above ORC_BAND_CAP, or a quadratic [.]_+ clamp met) (may be NULL) */
  uint64_t* signature; /* [h][w] hash of the composited ids, stop and clamp state (may be NULL) */
  int32_t* n_outcomes; /* [h][w] outcomes enumerated (1 without an orc_alt_out) (may be NULL) */
} orc_fwd_out;

typedef struct {
  const double* dl_dimage; /* [h][w][3] */
  double* d_means;         /* [n][3] overwritten */
  double* d_log_scales;    /* [n][3] */
  double* d_quats;         /* [n][4] */
  double* d_opacity_logits;/* [n] */
  double* d_sh;            /* [n][(d+1)^2][3] */
  uint8_t* fragile_gauss;  /* [n] bit ch: colour channel ch is within its FP32 error bound of the max(0, .)
                              clamp (may be NULL) */
  /* Optional [n]-shaped outputs like the gradients: the sum of the absolute values of every per-pixel term
   * chained through the absolute Jacobian. It is the scale of the rounding error an FP32 accumulation of
   * the same terms can make, whatever their cancellation; tests use it to bound that error. */
  double* s_means;
  double* s_log_scales;
  double* s_quats;
  double* s_opacity_logits;
  double* s_sh;
  /* Optional, likewise: the sum over the per-pixel terms of |term| times the bound of the relative error
   * of the GPU's FP32 pbar of that entry (the FP32 record and running sums; composite()), chained through
   * the absolute Jacobian: a bound of what the GPU's inputs, as opposed to its accumulation, put into
   * each gradient. */
  double* p_means;
  double* p_log_scales;
  double* p_quats;
  double* p_opacity_logits;
  double* p_sh;
} orc_bwd;

/* ------------------------------------------------------------------------------------------------
 * 1. Compositing operator over one ordered list (Eq. generalized_gaussian, Eq. nexp_p, Table 1).
 * ------------------------------------------------------------------------------------------------ */

/* Decisions near their thresholds. The GPU takes every compositing decision in FP32; where the FP64 value
 * lies within a bound of the FP32 error of its threshold, the GPU may legitimately go the other way. A
 * decider records such "borderline" decisions in the order the walk meets them and can take each of them
 * either way: path[j] = 1 takes the j-th borderline decision against its FP64 outcome. With path = NULL
 * every decision is the FP64 one. */
typedef struct {
  const uint8_t* path;
  int n_path;
  int n_seen; /* borderline decisions met in this walk */
} decider;

/* The FP64 outcome `choice` of a decision whose value lies at signed distance `dist` from its threshold,
 * with error bound `band` (>= 0) of the FP32 computation of that distance. */
static int decide(decider* d, int choice, double dist, double band) {
  if (!d || !(fabs(dist) <= band)) return choice;
  int j = d->n_seen++;
  return (j < d->n_path && d->path[j]) ? !choice : choice;
}

/* FP32 unit roundoff and the safety factor of the first-order error bounds below. */
#define U32 (1.0 / 16777216.0)
#define ORC_SAFETY 2.0
#define kLn2d 0.69314718055994530942

typedef struct {
  double alpha_min; /* candidates below it are skipped (0: every candidate is composited) */
  double alpha_max; /* alpha = min(alpha_max, raw) (> 1: no clamp) */
  double t_eps;     /* exponential stop (0: none) */
  int max_splats;   /* 0 = unlimited */
} comp_opts;

typedef struct {
  int m;            /* list entries composited (overdraw) */
  int saturated;    /* quadratic/blended: the ray saturated at composited entry m-1 (that entry is k) */
  double color[3];  /* L0, background included */
  double T_end;     /* Tbar after the composited entries */
  int clamp_fired;  /* the [.]_+ clamp of a quadratic slope term was active */
  int k_lin, k_exp; /* Vicini: composited entry where its linear list saturated / before which its
                       exponential list stopped (-1: none) */
} comp_result;

/* Composite candidates 0..n-1 front to back. raw[i] is the splat's aleph K(p) before the alpha_max clamp
 * (or the final alpha of a plain list), E[3 i..] its emission. band[i] (NULL: all decisions exact) is the
 * error bound of the FP32 log2(raw[i]) that the GPU compares; from it follow the bounds of the running
 * sums, propagated to first order and widened by ORC_SAFETY. Writes, for the composited entries j < m,
 * idx[j] (candidate index), alpha[j], clamped[j] (alpha_max clamp taken), pbar[j] and, when perr is not
 * NULL, perr[j]: the bound of the relative error of the GPU's FP32 pbar[j] (0 without bands). */
static void composite(int kind, double param, const comp_opts* co, const double bg[3], int n, const double* raw,
                      const double* band, const double* E, decider* d, int* idx, double* alpha, uint8_t* clamped,
                      double* pbar, double* perr, comp_result* r) {
  memset(r, 0, sizeof(*r));
  r->k_lin = r->k_exp = -1;
  double C[3] = {0, 0, 0};
  const double lmin = log2(co->alpha_min), lmax = log2(co->alpha_max);
  /* quadratic / blended / Vicini-linear: S = sum of slope terms, tau = sum of alphas, P = prod(1 - alpha);
   * exponential / Vicini-exponential: T = prod(1 - alpha). err_* are absolute error bounds of the FP32
   * values, relP and relT relative ones. */
  double S = 0.0, tau = 0.0, P = 1.0, T = 1.0, Ce[3] = {0, 0, 0};
  double err_S = 0.0, err_tau = 0.0, relP = 0.0, relT = 0.0;
  int sat = 0, stop_e = 0, m = 0;
  for (int i = 0; i < n; ++i) {
    if (co->max_splats > 0 && m == co->max_splats) break;
    /* the alpha test and the alpha_max clamp, both on log2(raw) */
    const double bl = band ? band[i] : 0.0, l2 = log2(raw[i]);
    if (!decide(band ? d : NULL, raw[i] >= co->alpha_min, l2 - lmin, bl)) continue;
    const int cl = decide(band ? d : NULL, raw[i] >= co->alpha_max, l2 - lmax, bl);
    const double a = cl ? co->alpha_max : raw[i];
    const double ea = cl ? 0.0 : kLn2d * bl; /* relative error bound of alpha */
    const double* Ei = &E[3 * i];
    double p, pe_rel = 0.0;
    int stop_here = 0, stop_before = 0;
    if (kind == ORC_EXP) {
      /* pbar_i = alpha_i T_i with T_i = prod_{j<i}(1 - alpha_j) (Table 1, row 1). The exponential never
       * reaches zero; the ray stops before the splat that would take T below t_eps. */
      const double testT = T * (1.0 - a);
      const double rel = relT + a * ea / (1.0 - a) + 2.0 * U32;
      if (co->t_eps > 0 && decide(d, testT < co->t_eps, testT - co->t_eps, ORC_SAFETY * rel * testT)) break;
      p = a * T;
      pe_rel = ea + relT + U32;
      T = testT;
      relT = rel;
    } else if (kind == ORC_QUAD || kind == ORC_BLEND) {
      /* pbar_i = slope term while the running sum stays below 1; the splat k whose slope term would reach
       * 1 gets the remainder 1 - sum_{j<k} pbar_j and the ray stops (Eq. nexp_p). */
      double pt, err_pt;
      if (kind == ORC_QUAD) {
        const double f = 1.0 + param * tau;
        const double err_f = fabs(param) * err_tau + U32 * fabs(f);
        if (decide(d, f < 0, f, ORC_SAFETY * err_f)) { r->clamp_fired = 1; pt = 0.0; err_pt = 0.0; }
        else { pt = a * f; err_pt = pt * (ea + U32) + a * err_f; }
      } else {
        const double f = 1.0 - param + param * P;
        pt = a * f;
        err_pt = pt * (ea + 2.0 * U32) + a * param * P * relP;
      }
      const double Sn = S + pt;
      const double err_Sn = err_S + err_pt + U32 * Sn;
      if (decide(d, Sn >= 1.0, Sn - 1.0, ORC_SAFETY * err_Sn)) {
        p = 1.0 - S;
        pe_rel = p > 0 ? (err_S + U32) / p : 0.0;
        sat = 1;
        stop_here = 1;
      } else {
        p = pt;
        pe_rel = pt > 0 ? err_pt / pt : 0.0;
        S = Sn;
        err_S = err_Sn;
        tau += a;
        err_tau += a * ea + U32 * tau;
        P *= 1.0 - a;
        relP += a * ea / (1.0 - a) + 2.0 * U32;
      }
    } else { /* ORC_VICINI: lerp of the saturated linear list and the exponential list */
      const double gam = param;
      double pe = 0.0, pl = 0.0;
      if (!stop_e) {
        const double testT = T * (1.0 - a);
        const double rel = relT + a * ea / (1.0 - a) + 2.0 * U32;
        if (co->t_eps > 0 && decide(d, testT < co->t_eps, testT - co->t_eps, ORC_SAFETY * rel * testT)) {
          stop_e = 1;
          r->k_exp = m;
        } else {
          pe = a * T;
          pe_rel = ea + relT + U32;
          T = testT;
          relT = rel;
        }
      }
      if (sat && stop_e) stop_before = 1; /* both lists have stopped before this splat */
      if (!stop_before) {
        if (!sat) {
          const double Sn = S + a, err_Sn = err_S + a * ea + U32 * Sn;
          if (decide(d, Sn >= 1.0, Sn - 1.0, ORC_SAFETY * err_Sn)) {
            pl = 1.0 - S;
            pe_rel = fmax(pe_rel, pl > 0 ? (err_S + U32) / pl : 0.0);
            S = 1.0;
            sat = 1;
            r->k_lin = m;
          } else {
            pl = a;
            pe_rel = fmax(pe_rel, ea);
            S = Sn;
            err_S = err_Sn;
          }
        }
        for (int ch = 0; ch < 3; ++ch) Ce[ch] += Ei[ch] * pe;
        p = (1.0 - gam) * pl + gam * pe;
        if (sat && stop_e) stop_here = 1;
      } else {
        p = 0.0;
      }
    }
    if (stop_before) break;
    idx[m] = i;
    alpha[m] = a;
    clamped[m] = (uint8_t)cl;
    pbar[m] = p;
    if (perr) perr[m] = band ? ORC_SAFETY * pe_rel : 0.0;
    for (int ch = 0; ch < 3; ++ch) C[ch] += Ei[ch] * p;
    ++m;
    if (stop_here) break;
  }
  r->m = m;
  r->saturated = (kind == ORC_QUAD || kind == ORC_BLEND) ? sat : 0;
  if (kind == ORC_EXP) r->T_end = T;
  else if (kind == ORC_VICINI) r->T_end = (1.0 - param) * (1.0 - S) + param * T;
  else r->T_end = sat ? 0.0 : 1.0 - S;
  for (int ch = 0; ch < 3; ++ch) r->color[ch] = C[ch] + bg[ch] * r->T_end;
}

/* Adjoint of composite() over its composited entries (alpha[j], E_j = E[3 j..], pbar[j], j < r->m): given
 * g = dL/dL0 (RGB), write dL/dalpha_j and dL/dE_j. */
static void composite_adjoint(int kind, double param, const double bg[3], const comp_result* r,
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
  } else { /* ORC_VICINI: (1 - gamma) x linear adjoint + gamma x exponential adjoint, each over its own list
            * with the stops the forward walk took (r->k_lin, r->k_exp) */
    double gam = param;
    double* d2 = (double*)malloc(sizeof(double) * (size_t)m);
    double* dE2 = (double*)malloc(sizeof(double) * 3 * (size_t)m);
    double* p2 = (double*)calloc((size_t)m, sizeof(double));
    comp_result rl, re;
    memset(&rl, 0, sizeof rl);
    memset(&re, 0, sizeof re);
    rl.m = r->k_lin >= 0 ? r->k_lin + 1 : m; /* linear part: saturates at k_lin, or never */
    rl.saturated = r->k_lin >= 0;
    composite_adjoint(ORC_QUAD, 0.0, bg, &rl, alpha, E, p2, g, d2, dE2);
    for (int i = 0; i < rl.m; ++i) dalpha[i] += (1.0 - gam) * d2[i];
    re.m = r->k_exp >= 0 ? r->k_exp : m; /* exponential part: stops before k_exp, or never */
    if (re.m > 0) {
      composite_adjoint(ORC_EXP, 0.0, bg, &re, alpha, E, p2, g, d2, dE2);
      for (int i = 0; i < re.m; ++i) dalpha[i] += gam * d2[i];
    }
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
 * plus (real only) the 2D covariance's largest eigenvalue, each colour channel's value before the
 * max(0, .) clamp and, when e_band is not NULL, the error bound of its FP32 computation (see below).
 * Bit ch of eflip takes channel ch's clamp against the sign of its value. Returns 0 when the splat cannot
 * be formed. */
static int project_c(const orc_camera* cam, double dilation, int K, const cplx* p, const cplx* s,
                     const cplx* q, cplx logit, const cplx* sh, cplx* rec, double* lam_max, double* e_real,
                     double* e_band, int eflip) {
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
    const int clamp = creal(e) < 0;
    rec[6 + ch] = (clamp ^ ((eflip >> ch) & 1)) ? 0.0 : e;
  }
  if (e_band) {
    /* FP32 error of the channel value: the direction d = (mean - camera centre) / |.| carries a relative
     * error of dd = u (3 + (|mean| + 4 |centre|) / |mean - centre|) (the centre is formed from R and t in
     * FP32); Y_lm of degree l is a degree-l polynomial in d (relative error l dd + 4 u), and the sum of
     * 1 + K terms adds 4 u of its absolute size. */
    double pm = 0, cm = 0, dist = cabs(dn);
    for (int j = 0; j < 3; ++j) { pm += creal(p[j]) * creal(p[j]); cm += cc[j] * cc[j]; }
    const double dd = U32 * (3.0 + (sqrt(pm) + 4.0 * sqrt(cm)) / dist);
    for (int ch = 0; ch < 3; ++ch) {
      double tot = 0.5, deg_err = 0;
      for (int k = 0; k < K; ++k) {
        const double t = cabs(Y[k]) * fabs(creal(sh[3 * k + ch]));
        const int l = k < 1 ? 0 : k < 4 ? 1 : k < 9 ? 2 : 3;
        tot += t;
        deg_err += t * l;
      }
      e_band[ch] = ORC_SAFETY * (8.0 * U32 * tot + dd * deg_err);
    }
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
  double e_real[3];  /* colour channels before the max(0, .) clamp */
  double e_band[3];  /* FP32 error bound of e_real */
  double pos_err[2]; /* FP32 error bound of (u, v), in units of U32 */
  double cand_r;     /* radius of the disc outside which alpha < alpha_min 2^-ORC_BAND_CAP */
  float z32;
  int valid;         /* in front of the near plane, aleph >= alpha_min */
  int cand;          /* in front of the near plane, aleph >= alpha_min 2^-ORC_BAND_CAP */
} splat_d;

/* Largest error bound (log2 units) given to an alpha decision; a larger bound marks the pixel unresolved. */
#define ORC_BAND_CAP 0.5

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
  if (!project_c(cam, o->dilation, K, p, s, q, sc->opacity_logits[g], sh, rec, &lam, out->e_real, out->e_band, 0))
    return;
  for (int j = 0; j < 9; ++j) out->rec[j] = creal(rec[j]);
  /* FP32 error of the screen position: the view transform (three fma per coordinate, error
   * 3 u (sum_j |R_rj p_j| + |t_r|)) scaled by f / z, the division by z (relative error of z likewise), the
   * products and the principal point: 4 u |u|. In units of u. */
  {
    const double* V = cam->viewmat;
    double ax[3], pv[3];
    for (int r = 0; r < 3; ++r) {
      ax[r] = fabs(V[4 * r + 3]);
      pv[r] = V[4 * r + 3];
      for (int j = 0; j < 3; ++j) {
        ax[r] += fabs(V[4 * r + j] * sc->means[3 * g + j]);
        pv[r] += V[4 * r + j] * sc->means[3 * g + j];
      }
    }
    const double fu[2] = {cam->fx, cam->fy};
    for (int t = 0; t < 2; ++t)
      out->pos_err[t] = 4.0 * fabs(out->rec[t]) + 3.0 * fu[t] / pv[2] * (ax[t] + fabs(pv[t] / pv[2]) * ax[2]);
  }
  double aleph = out->rec[5];
  const double cand_min = o->alpha_min * exp2(-ORC_BAND_CAP);
  if (!(aleph >= cand_min)) return; /* alpha = aleph K <= aleph stays below every candidate threshold */
  out->cand = 1;
  out->cand_r = sqrt(2.0 * log(aleph / cand_min) * lam);
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
  int32_t g;   /* local splat index */
  double raw;  /* aleph K(p) before the alpha_max clamp */
  double band; /* error bound of the GPU's FP32 log2(raw) */
} entry;

static int entry_cmp(const void* a, const void* b) {
  const entry* x = (const entry*)a;
  const entry* y = (const entry*)b;
  if (x->z32 < y->z32) return -1;
  if (x->z32 > y->z32) return 1;
  return (x->g > y->g) - (x->g < y->g);
}

/* FP32 error bound of log2(aleph K(p)) as the GPU forms it: L + dx (A' dx + B' dy) + C' dy^2 from a splat
 * record computed in FP32, then ex2. In units of u (to first order):
 *   record conic: A and C to 16 u relative, B to 16 u sqrt(A C) (the 2D covariance is a sum of squares
 *     plus the dilation; its determinant by Cauchy-Binet), so |dq| <= 3 * 16 u (sqrt(A)|dx| + sqrt(C)|dy|)^2,
 *     times log2(e)/2 in log2 units: 35 Q;
 *   screen position (pos_err): |dl| = log2(e) (|A dx + B dy| du + |B dx + C dy| dv);
 *   L = log2(sigmoid(logit)) and the evaluation of the sum: 8 + 4 |L| + 4 |l|;
 * all widened by ORC_SAFETY. The GPU's alpha test and alpha_max clamp compare this value. */
static double alpha_band(const splat_d* s, double dx, double dy, double l2) {
  const double A = s->rec[2], B = s->rec[3], C = s->rec[4];
  const double L = log2(s->rec[5]);
  const double Q = pow(sqrt(A) * fabs(dx) + sqrt(C) * fabs(dy), 2.0);
  const double pos = 1.4426950408889634 * (fabs(A * dx + B * dy) * s->pos_err[0] + fabs(B * dx + C * dy) * s->pos_err[1]);
  return ORC_SAFETY * U32 * (8.0 + 4.0 * fabs(L) + 4.0 * fabs(l2) + 35.0 * Q + pos);
}

/* Per-entry record-gradient terms: ORC_TERMS values per (pixel, composited entry), see entry_terms(). */
#define ORC_TERMS 27

/* Sparse outputs of a pixel with several outcomes (per worker thread, merged after the join). */
typedef struct {
  int64_t pix;
  int32_t outcome, overdraw;
  double img[3];
} alt_fwd_row;

typedef struct {
  int64_t pix;
  int32_t outcome, lid;
  double g[ORC_TERMS]; /* entry_terms() */
} alt_grad_row;

typedef struct {
  alt_fwd_row* f;
  size_t nf, cf;
  alt_grad_row* g;
  size_t ng, cg;
} alt_buf;

static void* grow(void* p, size_t* cap, size_t need, size_t elem) {
  if (need <= *cap) return p;
  size_t nc = *cap ? *cap : 256;
  while (nc < need) nc *= 2;
  *cap = nc;
  return realloc(p, nc * elem);
}

/* Outputs for pixels with several legitimate outcomes. A decision of the compositing walk whose FP64
 * value lies within its FP32 error bound (see composite() and alpha_band()) may go either way on the GPU;
 * the oracle enumerates every combination of such decisions (depth first, in walk order, at most
 * ORC_MAX_OUTCOMES per pixel, else the pixel is "unresolved"). The window's image, overdraw and the
 * gradients are those of outcome 0, the all-FP64 walk; the rows below give every outcome of every pixel
 * with more than one, so that a test can accept any of them. Arrays are allocated by orc_render and
 * released by orc_free_alt. */
typedef struct {
  int64_t n_fwd;
  int64_t* fwd_pix;      /* window pixel y w + x */
  int32_t* fwd_outcome;  /* 0 = the FP64 walk */
  int32_t* fwd_overdraw;
  double* fwd_image;     /* [n_fwd][3] */
  /* backward: the per-entry terms of the record gradient of each outcome (as accumulated per splat) */
  int64_t n_grad;
  int64_t* grad_pix;
  int32_t* grad_outcome;
  int32_t* grad_ju;      /* row of jac / jac_gid */
  double* grad_rec;      /* [n_grad][27]: the terms of entry_terms(): dL/d(u, v, A, B, C, aleph, E0, E1, E2),
                            their absolute values and their FP32 error bounds */
  int32_t n_params;      /* 11 + 3 K */
  int64_t n_jac;
  int64_t* jac_gid;      /* Gaussians named by the rows above */
  double* jac;           /* [n_jac][9][n_params]: d(record) / d(raw parameters), complex step */
  /* Gaussians with a colour channel within its FP32 error bound of the max(0, .) clamp */
  int64_t n_eflip;
  int64_t* eflip_gid;
  uint8_t* eflip_mask;   /* bit ch: channel ch is borderline */
  double* eflip_dJ;      /* [n_eflip][3][n_params]: row 6 + ch of the Jacobian with that clamp taken the
                            other way, minus the row of outcome 0 (zero for channels not borderline) */
  double* eflip_gE;      /* [n_eflip][3]: dL/dE_ch of the splat summed over the window (outcome 0) */
} orc_alt_out;

#define ORC_MAX_OUTCOMES 64
#define ORC_MAX_DECISIONS 24

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
  uint8_t* px_capped;    /* a candidate's error bound exceeded ORC_BAND_CAP */
  orc_fwd_out* fwd;
  orc_bwd* bwd;
  int want_alt;
  alt_buf* alt;          /* per thread */
  double* grad_rec;      /* per thread [nthreads][nloc][ORC_TERMS] */
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

/* Per-thread scratch of one pixel's walk. */
typedef struct {
  int cap;
  double *raw, *band, *E, *alpha, *pbar, *perr, *Ee, *dal, *dE;
  int* idx;
  uint8_t* clamped;
} walk_buf;

static void walk_reserve(walk_buf* b, int n) {
  if (n <= b->cap) return;
  b->cap = n;
  b->raw = (double*)realloc(b->raw, sizeof(double) * n);
  b->band = (double*)realloc(b->band, sizeof(double) * n);
  b->E = (double*)realloc(b->E, sizeof(double) * 3 * n);
  b->alpha = (double*)realloc(b->alpha, sizeof(double) * n);
  b->pbar = (double*)realloc(b->pbar, sizeof(double) * n);
  b->perr = (double*)realloc(b->perr, sizeof(double) * n);
  b->Ee = (double*)realloc(b->Ee, sizeof(double) * 3 * n);
  b->dal = (double*)realloc(b->dal, sizeof(double) * n);
  b->dE = (double*)realloc(b->dE, sizeof(double) * 3 * n);
  b->idx = (int*)realloc(b->idx, sizeof(int) * n);
  b->clamped = (uint8_t*)realloc(b->clamped, (size_t)n);
}

static void walk_free(walk_buf* b) {
  free(b->raw); free(b->band); free(b->E); free(b->alpha); free(b->pbar); free(b->perr); free(b->Ee); free(b->dal);
  free(b->dE); free(b->idx); free(b->clamped);
}

/* The terms of composited entry j of a walk at pixel (px, py), given dL/dalpha_j and dL/dE_j: out[0..9)
 * the 9 record-gradient terms dL/d(u, v, A, B, C, aleph, E0, E1, E2), out[9..18) their absolute values,
 * out[18..27) their absolute values times rel, the bound of the relative error of the GPU's FP32 pbar_j
 * (which is proportional to alpha_j: the error the FP32 record and running sums carry into the term). */
static void entry_terms(const splat_d* s, double px, double py, double a, int clamped, double dal,
                        const double* dE, double rel, double* out) {
  memset(out, 0, sizeof(double) * ORC_TERMS);
  for (int ch = 0; ch < 3; ++ch) {
    out[6 + ch] = dE[ch];
    out[15 + ch] = fabs(dE[ch]);
    out[24 + ch] = fabs(dE[ch]) * rel;
  }
  if (clamped) return; /* alpha = alpha_max does not depend on the splat */
  /* alpha = aleph exp(-q/2), q = A dx^2 + 2 B dx dy + C dy^2, (dx, dy) = p - (u, v) */
  double dx = px - s->rec[0], dy = py - s->rec[1];
  double A = s->rec[2], B = s->rec[3], C = s->rec[4];
  double q = A * dx * dx + 2.0 * B * dx * dy + C * dy * dy;
  double G = exp(-0.5 * q);
  double dq = dal * (-0.5 * a);
  double t[6] = {dq * (-2.0 * (A * dx + B * dy)), dq * (-2.0 * (B * dx + C * dy)), dq * dx * dx,
                 dq * 2.0 * dx * dy, dq * dy * dy, dal * G};
  for (int r = 0; r < 6; ++r) {
    out[r] = t[r];
    out[9 + r] = fabs(t[r]);
    out[18 + r] = fabs(t[r]) * rel;
  }
}

static void* render_rows(void* argp) {
  worker_arg* wa = (worker_arg*)argp;
  render_job* J = wa->job;
  const orc_window* w = J->win;
  int kind = J->model->kind;
  double par = J->model->param;
  double* grec = J->grad_rec ? J->grad_rec + (size_t)wa->tid * (size_t)J->nloc * ORC_TERMS : NULL;
  alt_buf* ab = J->alt ? &J->alt[wa->tid] : NULL;
  const comp_opts co = {J->o->alpha_min, J->o->alpha_max, J->o->t_eps, J->o->max_splats};
  walk_buf wb;
  memset(&wb, 0, sizeof wb);
  uint8_t paths[ORC_MAX_OUTCOMES][ORC_MAX_DECISIONS];
  int path_len[ORC_MAX_OUTCOMES];
  for (int yy = wa->tid; yy < w->h; yy += J->nthreads) {
    for (int xx = 0; xx < w->w; ++xx) {
      int64_t pix = (int64_t)yy * w->w + xx;
      entry* L = J->ent + J->start[pix];
      int n = (int)(J->start[pix + 1] - J->start[pix]);
      qsort(L, (size_t)n, sizeof(entry), entry_cmp);
      walk_reserve(&wb, n > 0 ? n : 1);
      int listed = 0;
      for (int i = 0; i < n; ++i) {
        wb.raw[i] = L[i].raw;
        wb.band[i] = L[i].band;
        listed += L[i].raw >= J->o->alpha_min;
        for (int ch = 0; ch < 3; ++ch) wb.E[3 * i + ch] = J->sp[L[i].g].rec[6 + ch];
      }
      if (J->fwd->n_listed) J->fwd->n_listed[pix] = listed;
      const double* g = J->bwd ? &J->bwd->dl_dimage[3 * pix] : NULL;
      const int want_grad = grec && !(g[0] == 0 && g[1] == 0 && g[2] == 0);
      const double px = J->win->x0 + xx + 0.5, py = J->win->y0 + yy + 0.5;
      /* depth-first enumeration of the borderline decisions; outcome 0 is the FP64 walk */
      int n_stack = 1, outcomes = 0, unresolved = J->px_capped[pix], border = 0;
      path_len[0] = 0;
      while (n_stack > 0) {
        --n_stack;
        uint8_t path[ORC_MAX_DECISIONS];
        const int plen = path_len[n_stack];
        memcpy(path, paths[n_stack], (size_t)plen);
        decider d = {path, plen, 0};
        comp_result r;
        composite(kind, par, &co, J->o->background, n, wb.raw, wb.band, wb.E, &d, wb.idx, wb.alpha, wb.clamped,
                  wb.pbar, wb.perr, &r);
        const int oc = outcomes++;
        if (oc == 0) {
          for (int ch = 0; ch < 3; ++ch) J->fwd->image[3 * pix + ch] = r.color[ch];
          J->fwd->overdraw[pix] = r.m;
          if (J->fwd->signature) {
            uint64_t h = 1469598103934665603ULL;
            for (int i = 0; i < r.m; ++i)
              h = fnv(h, (uint64_t)J->gid[L[wb.idx[i]].g] * 4 + (uint64_t)wb.clamped[i]);
            h = fnv(h, (uint64_t)r.m * 2 + (uint64_t)r.saturated);
            if (kind == ORC_VICINI) h = fnv(h, ((uint64_t)(r.k_lin + 1) << 32) | (uint64_t)(r.k_exp + 1));
            J->fwd->signature[pix] = h;
          }
          if (r.clamp_fired) unresolved = 1; /* the [.]_+ clamp: not reached for c >= -1/2 (Sec. 4.3) */
          border = d.n_seen > 0;
        }
        const int several = border && J->want_alt;
        /* children: take each borderline decision met after the path's own against its FP64 outcome */
        for (int j = d.n_seen - 1; j >= plen && J->want_alt; --j) {
          if (j >= ORC_MAX_DECISIONS || n_stack >= ORC_MAX_OUTCOMES) { unresolved = 1; continue; }
          memcpy(paths[n_stack], path, (size_t)plen);
          memset(paths[n_stack] + plen, 0, (size_t)(j - plen));
          paths[n_stack][j] = 1;
          path_len[n_stack] = j + 1;
          ++n_stack;
        }
        if (oc + 1 >= ORC_MAX_OUTCOMES && n_stack > 0) { unresolved = 1; n_stack = 0; }
        if (several && ab) {
          ab->f = (alt_fwd_row*)grow(ab->f, &ab->cf, ab->nf + 1, sizeof(alt_fwd_row));
          alt_fwd_row* fr = &ab->f[ab->nf++];
          fr->pix = pix;
          fr->outcome = oc;
          fr->overdraw = r.m;
          for (int ch = 0; ch < 3; ++ch) fr->img[ch] = r.color[ch];
        }
        if (!want_grad) continue;
        for (int i = 0; i < r.m; ++i)
          for (int ch = 0; ch < 3; ++ch) wb.Ee[3 * i + ch] = wb.E[3 * wb.idx[i] + ch];
        composite_adjoint(kind, par, J->o->background, &r, wb.alpha, wb.Ee, wb.pbar, g, wb.dal, wb.dE);
        if (several && ab) ab->g = (alt_grad_row*)grow(ab->g, &ab->cg, ab->ng + (size_t)r.m, sizeof(alt_grad_row));
        for (int i = 0; i < r.m; ++i) {
          const int lid = L[wb.idx[i]].g;
          double tt[ORC_TERMS];
          entry_terms(&J->sp[lid], px, py, wb.alpha[i], wb.clamped[i], wb.dal[i], &wb.dE[3 * i], wb.perr[i], tt);
          if (oc == 0) {
            double* gr = grec + (size_t)lid * ORC_TERMS;
            for (int k = 0; k < ORC_TERMS; ++k) gr[k] += tt[k];
          }
          if (several && ab) {
            alt_grad_row* gr = &ab->g[ab->ng++];
            gr->pix = pix;
            gr->outcome = oc;
            gr->lid = lid;
            memcpy(gr->g, tt, sizeof tt);
          }
        }
      }
      if (J->fwd->fragile) J->fwd->fragile[pix] = (uint8_t)(unresolved ? 2 : border ? 1 : 0);
      if (J->fwd->n_outcomes) J->fwd->n_outcomes[pix] = outcomes;
    }
  }
  walk_free(&wb);
  return NULL;
}

/* Complex-step chain from record gradients to raw-parameter gradients for one Gaussian (bit ch of eflip
 * takes colour channel ch's max(0, .) clamp the other way). */
static void chain_to_params(const orc_scene* sc, const orc_camera* cam, const orc_opts* o, int64_t g,
                            const double* grec, const double* gabs, const double* gerr, orc_bwd* b, int eflip) {
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
    double* pdst;
    int64_t at;
    if (j < 3) {
      p[j] += I * h;
      at = 3 * g + j;
      dst = &b->d_means[at]; sdst = b->s_means ? &b->s_means[at] : NULL; pdst = b->p_means ? &b->p_means[at] : NULL;
    } else if (j < 6) {
      s[j - 3] += I * h;
      at = 3 * g + j - 3;
      dst = &b->d_log_scales[at];
      sdst = b->s_log_scales ? &b->s_log_scales[at] : NULL;
      pdst = b->p_log_scales ? &b->p_log_scales[at] : NULL;
    } else if (j < 10) {
      q[j - 6] += I * h;
      at = 4 * g + j - 6;
      dst = &b->d_quats[at]; sdst = b->s_quats ? &b->s_quats[at] : NULL; pdst = b->p_quats ? &b->p_quats[at] : NULL;
    } else if (j == 10) {
      logit += I * h;
      dst = &b->d_opacity_logits[g];
      sdst = b->s_opacity_logits ? &b->s_opacity_logits[g] : NULL;
      pdst = b->p_opacity_logits ? &b->p_opacity_logits[g] : NULL;
    } else {
      sh[j - 11] += I * h;
      at = (int64_t)3 * K * g + j - 11;
      dst = &b->d_sh[at]; sdst = b->s_sh ? &b->s_sh[at] : NULL; pdst = b->p_sh ? &b->p_sh[at] : NULL;
    }
    if (!project_c(cam, o->dilation, K, p, s, q, logit, sh, rec, &lam, er, NULL, eflip)) continue;
    double acc = 0, sacc = 0, pacc = 0;
    for (int r = 0; r < 9; ++r) {
      const double jr = cimag(rec[r]) / h;
      acc += grec[r] * jr;
      if (gabs) sacc += gabs[r] * fabs(jr);
      if (gerr) pacc += gerr[r] * fabs(jr);
    }
    *dst = acc;
    if (sdst) *sdst = sacc;
    if (pdst) *pdst = pacc;
  }
}

/* Project every Gaussian: rec [n][10], z32 [n], valid [n]; pos_err [n][2] (the FP32 error bound of (u, v),
 * pixels) and e_band [n][3] (of the colour channels before the clamp) may be NULL. */
int orc_project(const orc_scene* sc, const orc_camera* cam, const orc_opts* o, double* rec, float* z32,
                int32_t* valid, double* pos_err, double* e_band) {
  for (int64_t g = 0; g < sc->n; ++g) {
    splat_d s;
    project_one(sc, cam, o, g, &s);
    memcpy(&rec[ORC_REC * g], s.rec, sizeof(s.rec));
    z32[g] = s.z32;
    valid[g] = s.valid;
    if (pos_err) { pos_err[2 * g] = s.pos_err[0] * U32; pos_err[2 * g + 1] = s.pos_err[1] * U32; }
    if (e_band) memcpy(&e_band[3 * g], s.e_band, sizeof(s.e_band));
  }
  return 0;
}

/* Jacobian of the record (u, v, A, B, C, aleph, E0, E1, E2) w.r.t. the raw parameters of Gaussian g,
 * [9][np] with np = 11 + 3 K, by complex step; eflip as in chain_to_params. */
int orc_project_jacobian(const orc_scene* sc, const orc_camera* cam, const orc_opts* o, int64_t g, double* jac,
                         int32_t eflip) {
  int K = sh_count(sc->sh_degree);
  int np = 11 + 3 * K;
  /* one Gaussian's slot of each gradient array: chain_to_params writes only index g */
  double dm[3], ds[3], dq[4], dl[1], dh[48];
  orc_bwd b;
  memset(&b, 0, sizeof(b));
  b.d_means = dm - 3 * g; b.d_log_scales = ds - 3 * g; b.d_quats = dq - 4 * g; b.d_opacity_logits = dl - g;
  b.d_sh = dh - (int64_t)3 * K * g;
  for (int r = 0; r < 9; ++r) {
    double e[9] = {0};
    e[r] = 1.0;
    memset(dm, 0, sizeof dm); memset(ds, 0, sizeof ds); memset(dq, 0, sizeof dq); dl[0] = 0; memset(dh, 0, sizeof dh);
    chain_to_params(sc, cam, o, g, e, NULL, NULL, &b, eflip);
    double* row = jac + (size_t)r * np;
    for (int t = 0; t < 3; ++t) row[t] = dm[t];
    for (int t = 0; t < 3; ++t) row[3 + t] = ds[t];
    for (int t = 0; t < 4; ++t) row[6 + t] = dq[t];
    row[10] = dl[0];
    for (int t = 0; t < 3 * K; ++t) row[11 + t] = dh[t];
  }
  return 0;
}

/* Jacobians of many Gaussians on pthreads (rows of orc_alt_out). */
typedef struct {
  const orc_scene* sc;
  const orc_camera* cam;
  const orc_opts* o;
  const int64_t* gids;
  int64_t n;
  double* jac;
  int np, nthreads, tid;
} jac_job;

static void* jac_rows(void* argp) {
  jac_job* J = (jac_job*)argp;
  for (int64_t i = J->tid; i < J->n; i += J->nthreads)
    orc_project_jacobian(J->sc, J->cam, J->o, J->gids[i], J->jac + (size_t)i * 9 * J->np, 0);
  return NULL;
}

static void jacobians(const orc_scene* sc, const orc_camera* cam, const orc_opts* o, const int64_t* gids, int64_t n,
                      int np, double* jac, int nthreads) {
  jac_job* jobs = (jac_job*)malloc(sizeof(jac_job) * nthreads);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
  for (int t = 0; t < nthreads; ++t) {
    jac_job j = {sc, cam, o, gids, n, jac, np, nthreads, t};
    jobs[t] = j;
    if (t > 0) pthread_create(&th[t], NULL, jac_rows, &jobs[t]);
  }
  jac_rows(&jobs[0]);
  for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(jobs);
  free(th);
}

void orc_free_alt(orc_alt_out* a) {
  if (!a) return;
  free(a->fwd_pix); free(a->fwd_outcome); free(a->fwd_overdraw); free(a->fwd_image);
  free(a->grad_pix); free(a->grad_outcome); free(a->grad_ju); free(a->grad_rec);
  free(a->jac_gid); free(a->jac);
  free(a->eflip_gid); free(a->eflip_mask); free(a->eflip_dJ); free(a->eflip_gE);
  memset(a, 0, sizeof(*a));
}

/* Render a window of the camera's image. brute_force = 1 tests every candidate splat at every pixel;
 * otherwise a splat is only tested at pixels whose centre lies in the bounding box of its candidate disc
 * (cand_r), outside of which alpha < alpha_min 2^-ORC_BAND_CAP holds by the eigenvalue bound
 * (project_one). alt (may be NULL) receives the outcomes of pixels with borderline decisions; with alt =
 * NULL they are only flagged. */
int orc_render(const orc_scene* sc, const orc_camera* cam, const orc_model* model, const orc_opts* o,
               const orc_window* win, int nthreads, int brute_force, orc_fwd_out* fwd, orc_bwd* bwd,
               orc_alt_out* alt) {
  if (nthreads < 1) nthreads = 1;
  if (alt) memset(alt, 0, sizeof(*alt));
  int64_t n = sc->n;
  int64_t npx = (int64_t)win->w * win->h;
  const double lmin = log2(o->alpha_min);
  /* project, keep the splats that can reach the window */
  splat_d* all = (splat_d*)malloc(sizeof(splat_d) * (size_t)(n > 0 ? n : 1));
  int64_t* gid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t nloc = 0;
  for (int64_t g = 0; g < n; ++g) {
    splat_d s;
    project_one(sc, cam, o, g, &s);
    if (!s.cand) continue;
    if (!brute_force) {
      double rb = s.cand_r + 1e-6;
      if (s.rec[0] + rb < win->x0 || s.rec[0] - rb > win->x0 + win->w) continue;
      if (s.rec[1] + rb < win->y0 || s.rec[1] - rb > win->y0 + win->h) continue;
    }
    all[nloc] = s;
    gid[nloc] = g;
    ++nloc;
  }
  /* gather: two passes (count, fill) over (splat, pixel) pairs; a candidate is a splat whose alpha is at
   * least alpha_min, or below it by no more than its FP32 error bound */
  int64_t* start = (int64_t*)calloc((size_t)npx + 1, sizeof(int64_t));
  uint8_t* capped = (uint8_t*)calloc((size_t)npx + 1, 1);
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
        double rb = s->cand_r + 1e-6;
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
          double l2 = log2(raw);
          if (!(l2 >= lmin - ORC_BAND_CAP)) continue;
          double band = alpha_band(s, dx, dy, l2);
          if (!(l2 >= lmin - band)) continue;
          int64_t pix = (int64_t)yy * win->w + xx;
          if (pass == 0) {
            start[pix + 1]++;
            if (band > ORC_BAND_CAP) capped[pix] = 1;
          } else {
            entry* e = &ent[cursor[pix]++];
            e->z32 = s->z32;
            e->g = (int32_t)l;
            e->raw = raw;
            e->band = band > ORC_BAND_CAP ? ORC_BAND_CAP : band;
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
  job.px_capped = capped; job.fwd = fwd; job.bwd = bwd; job.nthreads = nthreads;
  job.want_alt = alt != NULL;
  if (alt) job.alt = (alt_buf*)calloc((size_t)nthreads, sizeof(alt_buf));
  if (bwd) job.grad_rec = (double*)calloc((size_t)nthreads * (size_t)nloc * ORC_TERMS + 1, sizeof(double));
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
  worker_arg* wa = (worker_arg*)malloc(sizeof(worker_arg) * nthreads);
  for (int t = 0; t < nthreads; ++t) {
    wa[t].job = &job;
    wa[t].tid = t;
    if (t > 0) pthread_create(&th[t], NULL, render_rows, &wa[t]);
  }
  render_rows(&wa[0]);
  for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
  const int K = sh_count(sc->sh_degree);
  const int np = 11 + 3 * K;
  double* grec_sum = NULL;
  if (bwd) {
    memset(bwd->d_means, 0, sizeof(double) * 3 * (size_t)n);
    memset(bwd->d_log_scales, 0, sizeof(double) * 3 * (size_t)n);
    memset(bwd->d_quats, 0, sizeof(double) * 4 * (size_t)n);
    memset(bwd->d_opacity_logits, 0, sizeof(double) * (size_t)n);
    memset(bwd->d_sh, 0, sizeof(double) * 3 * (size_t)K * (size_t)n);
    if (bwd->fragile_gauss) memset(bwd->fragile_gauss, 0, (size_t)n);
    double* sarr[10] = {bwd->s_means, bwd->s_log_scales, bwd->s_quats, bwd->s_opacity_logits, bwd->s_sh,
                        bwd->p_means, bwd->p_log_scales, bwd->p_quats, bwd->p_opacity_logits, bwd->p_sh};
    size_t swid[5] = {3, 3, 4, 1, 3 * (size_t)K};
    for (int k = 0; k < 10; ++k)
      if (sarr[k]) memset(sarr[k], 0, sizeof(double) * swid[k % 5] * (size_t)n);
    grec_sum = (double*)calloc((size_t)nloc * ORC_TERMS + 1, sizeof(double));
    for (int64_t l = 0; l < nloc; ++l) {
      double* gr = grec_sum + (size_t)l * ORC_TERMS;
      for (int t = 0; t < nthreads; ++t)
        for (int r = 0; r < ORC_TERMS; ++r) gr[r] += job.grad_rec[((size_t)t * nloc + l) * ORC_TERMS + r];
      int nz = 0;
      for (int r = 0; r < ORC_TERMS; ++r) nz |= gr[r] != 0;
      if (!nz) continue;
      chain_to_params(sc, cam, o, gid[l], gr, gr + 9, gr + 18, bwd, 0);
      if (bwd->fragile_gauss)
        for (int ch = 0; ch < 3; ++ch)
          if (fabs(all[l].e_real[ch]) <= all[l].e_band[ch]) bwd->fragile_gauss[gid[l]] |= (uint8_t)(1 << ch);
    }
    free(job.grad_rec);
  }
  if (alt) {
    /* merge the threads' rows */
    size_t nf = 0, ng = 0;
    for (int t = 0; t < nthreads; ++t) { nf += job.alt[t].nf; ng += job.alt[t].ng; }
    alt->n_fwd = (int64_t)nf;
    alt->fwd_pix = (int64_t*)malloc(sizeof(int64_t) * (nf + 1));
    alt->fwd_outcome = (int32_t*)malloc(sizeof(int32_t) * (nf + 1));
    alt->fwd_overdraw = (int32_t*)malloc(sizeof(int32_t) * (nf + 1));
    alt->fwd_image = (double*)malloc(sizeof(double) * 3 * (nf + 1));
    alt->n_grad = (int64_t)ng;
    alt->grad_pix = (int64_t*)malloc(sizeof(int64_t) * (ng + 1));
    alt->grad_outcome = (int32_t*)malloc(sizeof(int32_t) * (ng + 1));
    alt->grad_ju = (int32_t*)malloc(sizeof(int32_t) * (ng + 1));
    alt->grad_rec = (double*)malloc(sizeof(double) * ORC_TERMS * (ng + 1));
    int32_t* ju_of = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nloc + 1));
    for (int64_t l = 0; l < nloc; ++l) ju_of[l] = -1;
    alt->jac_gid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nloc + 1));
    int64_t nj = 0;
    size_t kf = 0, kg = 0;
    for (int t = 0; t < nthreads; ++t) {
      alt_buf* b = &job.alt[t];
      for (size_t i = 0; i < b->nf; ++i, ++kf) {
        alt->fwd_pix[kf] = b->f[i].pix;
        alt->fwd_outcome[kf] = b->f[i].outcome;
        alt->fwd_overdraw[kf] = b->f[i].overdraw;
        memcpy(&alt->fwd_image[3 * kf], b->f[i].img, sizeof(double) * 3);
      }
      for (size_t i = 0; i < b->ng; ++i, ++kg) {
        const int32_t lid = b->g[i].lid;
        if (ju_of[lid] < 0) { ju_of[lid] = (int32_t)nj; alt->jac_gid[nj++] = gid[lid]; }
        alt->grad_pix[kg] = b->g[i].pix;
        alt->grad_outcome[kg] = b->g[i].outcome;
        alt->grad_ju[kg] = ju_of[lid];
        memcpy(&alt->grad_rec[ORC_TERMS * kg], b->g[i].g, sizeof(double) * ORC_TERMS);
      }
      free(b->f);
      free(b->g);
    }
    free(job.alt);
    free(ju_of);
    alt->n_params = np;
    alt->n_jac = nj;
    alt->jac = (double*)malloc(sizeof(double) * 9 * (size_t)np * (size_t)(nj + 1));
    jacobians(sc, cam, o, alt->jac_gid, nj, np, alt->jac, nthreads);
    /* colour channels near the clamp: the Jacobian rows with the clamp taken the other way */
    alt->eflip_gid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nloc + 1));
    alt->eflip_mask = (uint8_t*)malloc((size_t)(nloc + 1));
    alt->eflip_dJ = (double*)calloc(3 * (size_t)np * (size_t)(nloc + 1), sizeof(double));
    alt->eflip_gE = (double*)calloc(3 * (size_t)(nloc + 1), sizeof(double));
    int64_t ne = 0;
    for (int64_t l = 0; bwd && l < nloc; ++l) {
      int mask = 0;
      for (int ch = 0; ch < 3; ++ch)
        if (fabs(all[l].e_real[ch]) <= all[l].e_band[ch]) mask |= 1 << ch;
      if (!mask) continue;
      double* J0 = (double*)malloc(sizeof(double) * 9 * np);
      double* J1 = (double*)malloc(sizeof(double) * 9 * np);
      orc_project_jacobian(sc, cam, o, gid[l], J0, 0);
      orc_project_jacobian(sc, cam, o, gid[l], J1, mask);
      for (int ch = 0; ch < 3; ++ch) {
        if (!((mask >> ch) & 1)) continue;
        for (int t = 0; t < np; ++t)
          alt->eflip_dJ[((size_t)ne * 3 + ch) * np + t] = J1[(6 + ch) * np + t] - J0[(6 + ch) * np + t];
        alt->eflip_gE[3 * ne + ch] = grec_sum[(size_t)l * ORC_TERMS + 6 + ch];
      }
      free(J0);
      free(J1);
      alt->eflip_gid[ne] = gid[l];
      alt->eflip_mask[ne] = (uint8_t)mask;
      ++ne;
    }
    alt->n_eflip = ne;
  }
  free(grec_sum);
  free(th); free(wa); free(all); free(gid); free(start); free(capped); free(ent);
  return 0;
}

/* The compositing operator alone over one list (no geometry, no alpha_min filter, no alpha_max clamp):
 * pbar[0..n) (zeros past the stop), and out4 = {color r, g, b, T_end}; returns m. With g != NULL also
 * writes the adjoint. */
int orc_composite_list(int32_t kind, double param, double t_eps, int32_t max_splats, const double* bg, int32_t n,
                       const double* alpha, const double* E, double* pbar, double* out4, int32_t* saturated,
                       const double* g, double* dalpha, double* dE) {
  const comp_opts co = {0.0, INFINITY, t_eps, max_splats};
  int cap = n > 0 ? n : 1;
  int* idx = (int*)malloc(sizeof(int) * cap);
  double* a = (double*)malloc(sizeof(double) * cap);
  uint8_t* cl = (uint8_t*)malloc((size_t)cap);
  double* pb = (double*)malloc(sizeof(double) * cap);
  for (int i = 0; i < n; ++i) pbar[i] = 0;
  comp_result r;
  composite(kind, param, &co, bg, n, alpha, NULL, E, NULL, idx, a, cl, pb, NULL, &r);
  for (int j = 0; j < r.m; ++j) pbar[idx[j]] = pb[j];
  for (int ch = 0; ch < 3; ++ch) out4[ch] = r.color[ch];
  out4[3] = r.T_end;
  if (saturated) *saturated = r.saturated;
  if (g) {
    double* Ee = (double*)calloc(3 * (size_t)cap, sizeof(double));
    double* da = (double*)calloc((size_t)cap, sizeof(double));
    double* de = (double*)calloc(3 * (size_t)cap, sizeof(double));
    for (int j = 0; j < r.m; ++j)
      for (int ch = 0; ch < 3; ++ch) Ee[3 * j + ch] = E[3 * idx[j] + ch];
    composite_adjoint(kind, param, bg, &r, a, Ee, pb, g, da, de);
    for (int i = 0; i < n; ++i) { dalpha[i] = 0; dE[3 * i] = dE[3 * i + 1] = dE[3 * i + 2] = 0; }
    for (int j = 0; j < r.m; ++j) {
      dalpha[idx[j]] = da[j];
      for (int ch = 0; ch < 3; ++ch) dE[3 * idx[j] + ch] = de[3 * j + ch];
    }
    free(Ee); free(da); free(de);
  }
  free(idx); free(a); free(cl); free(pb);
  return r.m;
}

/* Every outcome of one list's walk (the enumeration orc_render runs per pixel): candidates raw[0..n) with
 * log2-domain error bounds band[0..n) (NULL: exact), the alpha_min filter and alpha_max clamp. Writes up
 * to max_out outcomes: m[o], out4[o][4] = {color, T_end}, pbar[o][n] (by candidate index; 0 where not
 * composited); returns their number, or -1 when there were more. Outcome 0 is the FP64 walk. */
int32_t orc_composite_outcomes(int32_t kind, double param, double alpha_min, double alpha_max, double t_eps,
                               int32_t max_splats, const double* bg, int32_t n, const double* raw, const double* band,
                               const double* E, int32_t max_out, int32_t* m_out, double* out4, double* pbar_out) {
  const comp_opts co = {alpha_min, alpha_max, t_eps, max_splats};
  int cap = n > 0 ? n : 1;
  int* idx = (int*)malloc(sizeof(int) * cap);
  double* a = (double*)malloc(sizeof(double) * cap);
  uint8_t* cl = (uint8_t*)malloc((size_t)cap);
  double* pb = (double*)malloc(sizeof(double) * cap);
  uint8_t paths[ORC_MAX_OUTCOMES][ORC_MAX_DECISIONS];
  int plen_of[ORC_MAX_OUTCOMES];
  int n_stack = 1, count = 0, over = 0;
  plen_of[0] = 0;
  while (n_stack > 0) {
    --n_stack;
    uint8_t path[ORC_MAX_DECISIONS];
    const int plen = plen_of[n_stack];
    memcpy(path, paths[n_stack], (size_t)plen);
    decider d = {path, plen, 0};
    comp_result r;
    composite(kind, param, &co, bg, n, raw, band, E, band ? &d : NULL, idx, a, cl, pb, NULL, &r);
    if (count >= max_out || count >= ORC_MAX_OUTCOMES) { over = 1; break; }
    m_out[count] = r.m;
    for (int ch = 0; ch < 3; ++ch) out4[4 * count + ch] = r.color[ch];
    out4[4 * count + 3] = r.T_end;
    for (int i = 0; i < n; ++i) pbar_out[(size_t)count * n + i] = 0;
    for (int j = 0; j < r.m; ++j) pbar_out[(size_t)count * n + idx[j]] = pb[j];
    ++count;
    for (int j = d.n_seen - 1; j >= plen; --j) {
      if (j >= ORC_MAX_DECISIONS || n_stack >= ORC_MAX_OUTCOMES) { over = 1; continue; }
      memcpy(paths[n_stack], path, (size_t)plen);
      memset(paths[n_stack] + plen, 0, (size_t)(j - plen));
      paths[n_stack][j] = 1;
      plen_of[n_stack] = j + 1;
      ++n_stack;
    }
  }
  free(idx); free(a); free(cl); free(pb);
  return over ? -1 : count;
}
