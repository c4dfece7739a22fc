// Per-tile front-to-back compositing (forward) and its path-replay adjoint (backward).
//
// One CTA per screen tile of any view of the batch (global tile index -> view by binary search over the
// views' first tiles), or persistent CTAs over a work list. The tile's depth-sorted splat list is walked in
// chunks of records staged in shared memory (half, one or two per pixel).
// Replay, and the forward of the exponential model (and of the quadratic ones on tiles of >= 256 pixels):
// two pixels per thread, (x, y) and (x, y + 4), so that a warp covers an 8 x 8 block; the two step through
// each entry together in packed FP32x2 instructions (add / mul / fma .rn.f32x2), each lane rounding like
// the one-pixel form, with the splat operands staged in duplicated pairs. The replay reduces both pixels'
// contributions once per 64 pixels. Other forwards: one thread per pixel, warps on 8 x 4 pixel blocks
// whose pixels are close and tend to saturate together.
//
// Forward, per pixel (Eq. generalized_gaussian with pbar_i from Eq. nexp_p and Table 1):
//   alpha_i = min(alpha_max, aleph_i K_i(p)), skipped when alpha_i < alpha_min;
//   quadratic:   pt = [alpha_i (1 + c taubar_i)]_+; if S + pt >= 1 the splat is k: pbar_k = 1 - S, the
//                ray has saturated and stops; else pbar_i = pt, S += pt, taubar += alpha_i;
//   exponential: stop before the splat that would take T below t_eps; pbar_i = alpha_i T, T *= 1 - alpha_i;
//   blended:     as quadratic with pt = alpha_i (1 - g + g P_i), P_i = prod_{j<i}(1 - alpha_j);
//   Vicini:      pbar_i = (1 - g) pbar_i^lin + g pbar_i^exp, the linear list saturating and the exponential
//                list stopping on their own; the ray stops once both have.
// A warp whose 32 pixels have all stopped leaves the chunk loop (ballot), and the CTA leaves the tile once
// every pixel has stopped (__syncthreads_count), which is where the faster-than-exponential models win.
//
// Backward (App. C), per pixel, replaying the same list front to back with identical FP32 arithmetic:
//   quadratic:   dL0/dalpha_i = DeltaE_i (1 + c taubar_i) + c Theta_i for i < k, Theta running down from
//                Theta_{-1} = A - E_k taubar_k (A = sum_{i<k} E_i alpha_i saved by the forward pass);
//                dL0/dE_i = pbar_i; dL0/dalpha_k = 0;
//   exponential: dL0/dalpha_i = T_i E_i - R_i / (1 - alpha_i), R_i = L0 - sum_{j<=i} E_j pbar_j;
//   blended:     dL0/dalpha_i = DeltaE_i (1 - g + g P_i) - g (B - B_i) / (1 - alpha_i), B_i the prefix sums
//                of DeltaE_l alpha_l P_l and B their total (saved by the forward pass);
//   Vicini:      (1 - g) x the linear adjoint + g x the exponential adjoint, each over its own list;
// then w = dL/d(log2 alpha) and its moments w, w dx, w dy, w dx^2, w dx dy, w dy^2 (which determine the
// gradient of the splat record, see the projection backward) and dL/dE: added to the per-Gaussian buffer by
// each lane that hit the splat when at most kDirectLanes did, else reduced over the warp with shuffles and
// added with one atomic-add instruction per value.
#include <algorithm>

#include <type_traits>

#include "ngs_internal.cuh"

namespace ngs {
namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;

// Stage splat record `id` in shared memory. An index outside [0, n_records) (which a correct binning never
// produces) is not read: the entry gets log2(aleph) = -inf, so no pixel composites it, and
// the device error word records the event.
__device__ __forceinline__ void stage_record(const float4* __restrict__ rec, uint32_t id, const RenderParams& rp,
                                             float4& r0, float4& r1, float& e2) {
  if (id < rp.n_records) {
    r0 = rec[3 * (size_t)id];
    r1 = rec[3 * (size_t)id + 1];
    e2 = rec[3 * (size_t)id + 2].x;
  } else {
    r0 = make_float4(0.f, 0.f, 0.f, 0.f);
    r1 = make_float4(0.f, -INFINITY, 0.f, 0.f);
    e2 = 0.f;
    atomicOr(rp.check, kCheckIndex);
  }
}

template <int TW, int TH, int PPT>
struct TileGeom {
  static constexpr int kPix = PPT;  // pixels per thread
  static constexpr int kThreads = TW * TH / kPix;
  static constexpr int kWarpsX = TW / 8;
  static_assert(TW % 8 == 0 && TH % (4 * PPT) == 0, "tile must be a multiple of 8 x (4 PPT)");
  // warp w covers the 8 x (4 PPT) block (w % kWarpsX, w / kWarpsX) of the tile; lane l owns its pixels
  // (l & 7, (l >> 3) + 4 k), k < PPT
  __device__ static void pixel(int tid, int k, int tile_x0, int tile_y0, int& x, int& y) {
    int warp = tid >> 5, lane = tid & 31;
    x = tile_x0 + (warp % kWarpsX) * 8 + (lane & 7);
    y = tile_y0 + (warp / kWarpsX) * 4 * PPT + (lane >> 3) + 4 * k;
  }
};

// The forward keeps one pixel per thread (a thread retires with its pixel); the replay takes two, so that
// the warp reduces once per 64 pixels.
constexpr int kBwdPix = 2;
// Replay: a splat hit by at most this many lanes of a warp is added by those lanes directly; more go through
// the warp reduction (32 atomics on one address serialise). Measured on GB300 with the packed replay at
// 500k Gaussians / 1080p: on 8x8 tiles 16 beats 8, 12, 24 and 32 (exponential replay 0.351 ms against
// 0.379 at 24 and 0.80 at 32), on 16x16 tiles 16 and 24 tie.
constexpr int kDirectLanes = 16;

// ---- forward ---------------------------------------------------------------------------------------

// Shared-memory staging of one chunk of CH splat records.
template <int CH>
struct StageBuf {
  float4 r0[CH];
  float4 r1[CH];
  float e2[CH];
};

// Stage list entries [base, base + CH) of the tile (those below `end`): slot k by thread k mod B.
template <int B, int CH>
__device__ __forceinline__ void stage_chunk(const float4* __restrict__ rec, const uint32_t* __restrict__ ids,
                                            const RenderParams& rp, uint32_t base, uint32_t end, StageBuf<CH>& sb,
                                            uint32_t* s_id) {
#pragma unroll
  for (int k = 0; k < (CH + B - 1) / B; ++k) {
    const int slot = k * B + (int)threadIdx.x;
    const uint32_t i = base + (uint32_t)slot;
    if (slot < CH && i < end) {
      const uint32_t id = ids[i];
      if (s_id) s_id[slot] = id < rp.n_records ? id : 0u;
      stage_record(rec, id, rp, sb.r0[slot], sb.r1[slot], sb.e2[slot]);
    }
  }
}

// Persistent schedule: the next tile of a CTA, the next entry of the work list taken with one atomic per
// CTA. Returns n_tiles when none is left.
__device__ __forceinline__ uint32_t next_tile(const uint32_t* __restrict__ work, uint32_t* counter, uint32_t n_tiles,
                                              uint32_t* s_next) {
  __syncthreads();  // every thread has read the previous s_next and is done with the staging buffers
  if (threadIdx.x == 0) *s_next = atomicAdd(counter, 1u);
  __syncthreads();
  const uint32_t w = *s_next;
  return w < n_tiles ? (work ? work[w] : w) : n_tiles;
}

// Staging of one chunk for the packed (two pixels per thread) forward and replay: every per-splat operand
// duplicated, so one 16-byte shared load gives the operand pairs {a, a, b, b} of two FP32x2 instructions.
template <int CH>
struct PairStageBuf {
  float4 q0[CH];  // {-u, -u, -v, -v}
  float4 q1[CH];  // {A', A', B', B'}
  float4 q2[CH];  // {C', C', L, L}
  float4 q3[CH];  // {E0, E0, E1, E1}
  float4 q4[CH];  // {E2, E2, record index (bits), 0}: one 16-byte load gives E2 and the atomics' target
};

// The packed form (exponential and quadratic models) is used while its staging (72 B per record) stays
// within 40 KB of static shared memory.
template <int KIND, int CH>
constexpr bool kPairForm = (KIND == NGS_MODEL_EXP || KIND == NGS_MODEL_QUAD) && sizeof(PairStageBuf<CH>) <= 40960;

template <int B, int CH>
__device__ __forceinline__ void stage_chunk_pairs(const float4* __restrict__ rec, const uint32_t* __restrict__ ids,
                                                  const RenderParams& rp, uint32_t base, uint32_t end,
                                                  PairStageBuf<CH>& sb) {
#pragma unroll
  for (int k = 0; k < (CH + B - 1) / B; ++k) {
    const int slot = k * B + (int)threadIdx.x;
    const uint32_t i = base + (uint32_t)slot;
    if (slot < CH && i < end) {
      const uint32_t id = ids[i];
      float4 r0, r1;
      float e2;
      stage_record(rec, id, rp, r0, r1, e2);
      sb.q0[slot] = make_float4(-r0.x, -r0.x, -r0.y, -r0.y);
      sb.q1[slot] = make_float4(r0.z, r0.z, r0.w, r0.w);
      sb.q2[slot] = make_float4(r1.x, r1.x, r1.y, r1.y);
      sb.q3[slot] = make_float4(r1.z, r1.z, r1.w, r1.w);
      sb.q4[slot] = make_float4(e2, e2, __uint_as_float(id < rp.n_records ? id : 0u), 0.f);
    }
  }
}

__device__ __forceinline__ float2 lo_hi(float4 q, bool hi) { return hi ? make_float2(q.z, q.w) : make_float2(q.x, q.y); }

template <int TW, int TH, int KIND, int CH>
__device__ __forceinline__ void forward_tile(const float4* __restrict__ rec, const uint32_t* __restrict__ ids,
                                             const uint2* __restrict__ ranges, const RenderParams& rp,
                                             const ViewParams* __restrict__ views, float* __restrict__ image,
                                             int32_t* __restrict__ overdraw, float4* __restrict__ state,
                                             uint32_t tile, StageBuf<CH>& sb) {
  using G = TileGeom<TW, TH, 1>;
  constexpr int B = G::kThreads;
  const TileView tv = tile_view(rp, views, (uint32_t)tile);
  const int W = tv.W, H = tv.H;
  const int tx = tv.local % tv.tiles_x, ty = tv.local / tv.tiles_x;
  int tid = threadIdx.x;
  int x, y;
  G::pixel(tid, 0, tx * TW, ty * TH, x, y);
  bool inside = x < W && y < H;
  float px = (float)x + 0.5f, py = (float)y + 0.5f;
  uint2 range = ranges[tile];
  bool done = !inside;
  int od = 0;
  uint32_t stop = range.y - range.x;  // entries walked (n of the replay state)
  bool saturated = false;  // quadratic / blended: the ray saturated; Vicini: its linear list did
  float C0 = 0.f, C1 = 0.f, C2 = 0.f;  // Vicini: the linear list's sum
  // quadratic (A = sum E alpha, tau) and blended (A = sum E alpha P, X = sum alpha P, P) state
  float S = 0.f, tau = 0.f, A0 = 0.f, A1 = 0.f, A2 = 0.f, Ek0 = rp.bg[0], Ek1 = rp.bg[1], Ek2 = rp.bg[2];
  float P = 1.f, X = 0.f;
  // exponential state (Vicini: its exponential list, with its own colour sum)
  float T = 1.f;
  bool stop_e = false;
  float Ce0 = 0.f, Ce1 = 0.f, Ce2 = 0.f;
  const float amax = rp.alpha_max, l2min = rp.log2_alpha_min, c = rp.c;
  for (uint32_t base = range.x; base < range.y; base += CH) {
    if (__syncthreads_count(done) == B) break;
    stage_chunk<B, CH>(rec, ids, rp, base, range.y, sb, nullptr);
    __syncthreads();
    int cnt = (int)min((uint32_t)CH, range.y - base);
    if (__any_sync(kFull, !done)) {
      for (int j = 0; j < cnt && !done; ++j) {
        float4 r0 = sb.r0[j], r1 = sb.r1[j];
        float dx, dy;
        float e = splat_log2_alpha(px, py, r0, r1, dx, dy);
        if (e < l2min) continue;
        float alpha = fminf(amax, fast_exp2(e));
        float E0 = r1.z, E1 = r1.w, E2 = sb.e2[j];
        if constexpr (KIND == NGS_MODEL_QUAD || KIND == NGS_MODEL_BLEND) {
          const float pt = KIND == NGS_MODEL_QUAD ? quad_slope(alpha, c, tau) : blend_slope(alpha, c, rp.c1, P);
          float Sn = __fadd_rn(S, pt);
          ++od;
          if (Sn >= 1.0f) {  // the saturating splat k: pbar_k = 1 - S (Eq. nexp_p)
            float pk = 1.0f - S;
            C0 = fmaf(E0, pk, C0);
            C1 = fmaf(E1, pk, C1);
            C2 = fmaf(E2, pk, C2);
            Ek0 = E0;
            Ek1 = E1;
            Ek2 = E2;
            saturated = true;
            done = true;
            stop = base + j + 1 - range.x;
            break;
          }
          C0 = fmaf(E0, pt, C0);
          C1 = fmaf(E1, pt, C1);
          C2 = fmaf(E2, pt, C2);
          const float w = KIND == NGS_MODEL_QUAD ? alpha : __fmul_rn(alpha, P);
          A0 = fmaf(E0, w, A0);
          A1 = fmaf(E1, w, A1);
          A2 = fmaf(E2, w, A2);
          S = Sn;
          if (KIND == NGS_MODEL_QUAD) {
            tau = __fadd_rn(tau, alpha);
          } else {
            X = __fadd_rn(X, w);
            P = __fmul_rn(P, __fsub_rn(1.0f, alpha));
          }
        } else if constexpr (KIND == NGS_MODEL_VICINI) {
          // the exponential list (own t_eps stop) and the linear list (own saturation), lerped by gamma
          float pe = 0.f;
          if (!stop_e) {
            const float testT = __fmul_rn(T, __fsub_rn(1.0f, alpha));
            if (testT < rp.t_eps) {
              stop_e = true;
            } else {
              pe = alpha * T;
              T = testT;
            }
          }
          if (saturated && stop_e) {  // both lists have stopped before this splat
            done = true;
            stop = base + j - range.x;
            break;
          }
          float pl = 0.f;
          if (!saturated) {
            const float Sn = __fadd_rn(S, alpha);
            if (Sn >= 1.0f) {
              pl = 1.0f - S;
              S = 1.0f;
              saturated = true;
              Ek0 = E0;
              Ek1 = E1;
              Ek2 = E2;
            } else {
              pl = alpha;
              S = Sn;
            }
          }
          C0 = fmaf(E0, pl, C0);
          C1 = fmaf(E1, pl, C1);
          C2 = fmaf(E2, pl, C2);
          Ce0 = fmaf(E0, pe, Ce0);
          Ce1 = fmaf(E1, pe, Ce1);
          Ce2 = fmaf(E2, pe, Ce2);
          ++od;
          if (saturated && stop_e) {
            done = true;
            stop = base + j + 1 - range.x;
            break;
          }
        } else {
          float testT = __fmul_rn(T, __fsub_rn(1.0f, alpha));
          if (testT < rp.t_eps) {
            done = true;
            stop = base + j - range.x;
            break;
          }
          float w = alpha * T;
          C0 = fmaf(E0, w, C0);
          C1 = fmaf(E1, w, C1);
          C2 = fmaf(E2, w, C2);
          T = testT;
          ++od;
        }
        if (rp.max_splats > 0 && od == rp.max_splats) {
          done = true;
          stop = base + j + 1 - range.x;
          break;
        }
      }
    }
  }
  if (!inside) return;  // (the caller's next barrier is reached by every thread)
  const size_t lpix = (size_t)y * W + x;                         // pixel within the view
  const size_t pix = view_pix_base(rp, views, tv.view) + lpix;  // packed pixel of the replay state
  float* const out_image = view_image(rp, views, tv.view, image);
  int32_t* const out_overdraw = view_overdraw(rp, views, tv.view, overdraw);
  float L0, L1, L2, Tend;
  if constexpr (KIND == NGS_MODEL_VICINI) {
    Tend = fmaf(rp.c1, 1.0f - S, c * T);  // lerp(1 - S, T_exp, gamma)
    L0 = fmaf(rp.c1, C0, fmaf(c, Ce0, rp.bg[0] * Tend));
    L1 = fmaf(rp.c1, C1, fmaf(c, Ce1, rp.bg[1] * Tend));
    L2 = fmaf(rp.c1, C2, fmaf(c, Ce2, rp.bg[2] * Tend));
  } else {
    Tend = KIND == NGS_MODEL_EXP ? T : (saturated ? 0.f : 1.f - S);
    L0 = C0 + rp.bg[0] * Tend;
    L1 = C1 + rp.bg[1] * Tend;
    L2 = C2 + rp.bg[2] * Tend;
  }
  out_image[3 * lpix] = L0;
  out_image[3 * lpix + 1] = L1;
  out_image[3 * lpix + 2] = L2;
  if (out_overdraw) out_overdraw[lpix] = od;
  uint32_t nbits = stop | (saturated ? 0x80000000u : 0u);
  if constexpr (KIND == NGS_MODEL_QUAD) {
    state[2 * pix] = make_float4(__uint_as_float(nbits), Ek0, Ek1, Ek2);
    state[2 * pix + 1] = make_float4(A0, A1, A2, tau);
  } else if constexpr (KIND == NGS_MODEL_BLEND) {
    state[2 * pix] = make_float4(__uint_as_float(nbits), Ek0, Ek1, Ek2);
    state[2 * pix + 1] = make_float4(A0, A1, A2, X);
  } else if constexpr (KIND == NGS_MODEL_VICINI) {
    state[2 * pix] = make_float4(__uint_as_float(nbits), Ek0, Ek1, Ek2);
    state[2 * pix + 1] = make_float4(fmaf(rp.bg[0], T, Ce0), fmaf(rp.bg[1], T, Ce1), fmaf(rp.bg[2], T, Ce2), 0.f);
  } else {
    state[2 * pix] = make_float4(__uint_as_float(nbits), L0, L1, L2);
    state[2 * pix + 1] = make_float4(Tend, 0.f, 0.f, 0.f);
  }
}

// Packed forward (exponential and quadratic): two pixels per thread, (x, y) and (x, y + 4), stepping through
// each entry together in FP32x2 instructions. Each lane rounds exactly like the one-pixel form above, so
// the image, the stop index and the replay state are the same bits. A pixel that has stopped, or that
// does not composite the entry, gets alpha = 0, which leaves its sums exactly unchanged.
template <int TW, int TH, int KIND, int CH>
__device__ __forceinline__ void forward_tile_pairs(const float4* __restrict__ rec, const uint32_t* __restrict__ ids,
                                                   const uint2* __restrict__ ranges, const RenderParams& rp,
                                                   const ViewParams* __restrict__ views, float* __restrict__ image,
                                                   int32_t* __restrict__ overdraw, float4* __restrict__ state,
                                                   uint32_t tile, PairStageBuf<CH>& sb) {
  using G = TileGeom<TW, TH, 2>;
  constexpr int B = G::kThreads;
  const TileView tv = tile_view(rp, views, (uint32_t)tile);
  const int W = tv.W, H = tv.H;
  const int tx = tv.local % tv.tiles_x, ty = tv.local / tv.tiles_x;
  int x, y;
  G::pixel(threadIdx.x, 0, tx * TW, ty * TH, x, y);  // the second pixel is (x, y + 4)
  const bool in0 = x < W && y < H, in1 = x < W && y + 4 < H;
  const float2 one = make_float2(1.f, 1.f), neg = make_float2(-1.f, -1.f), zero = make_float2(0.f, 0.f);
  const float2 px = make_float2((float)x + 0.5f, (float)x + 0.5f);
  const float2 py = make_float2((float)y + 0.5f, (float)(y + 4) + 0.5f);
  const uint2 range = ranges[tile];
  bool done0 = !in0, done1 = !in1;
  int od0 = 0, od1 = 0;
  uint32_t stop0 = range.y - range.x, stop1 = stop0;  // entries walked (n of the replay state)
  bool sat0 = false, sat1 = false;
  float2 C0 = zero, C1 = zero, C2 = zero;
  float2 S = zero, tau = zero, A0 = zero, A1 = zero, A2 = zero;  // quadratic
  float Ek[2][3] = {{rp.bg[0], rp.bg[1], rp.bg[2]}, {rp.bg[0], rp.bg[1], rp.bg[2]}};
  float2 T = one;  // exponential
  const float amax = rp.alpha_max, l2min = rp.log2_alpha_min;
  const float2 c2 = make_float2(rp.c, rp.c);
  for (uint32_t base = range.x; base < range.y; base += CH) {
    if (__syncthreads_count(done0 && done1) == B) break;
    stage_chunk_pairs<B, CH>(rec, ids, rp, base, range.y, sb);
    __syncthreads();
    const int cnt = (int)min((uint32_t)CH, range.y - base);
    if (__any_sync(kFull, !(done0 && done1))) {
      for (int j = 0; j < cnt; ++j) {
        const float4 q0 = sb.q0[j], q1 = sb.q1[j], q2 = sb.q2[j];
        const float2 dx = __fadd2_rn(px, lo_hi(q0, false));
        const float2 adx = __fmul2_rn(lo_hi(q1, false), dx);
        const float2 dy = __fadd2_rn(py, lo_hi(q0, true));
        const float2 t = __ffma2_rn(lo_hi(q1, true), dy, adx);
        const float2 cdd = __fmul2_rn(__fmul2_rn(lo_hi(q2, false), dy), dy);
        const float2 e = __fadd2_rn(lo_hi(q2, true), __ffma2_rn(dx, t, cdd));
        const bool on0 = !done0 && e.x >= l2min, on1 = !done1 && e.y >= l2min;
        // warp-uniform: a lane that does not composite the entry (or has stopped) runs the step with
        // alpha = 0, which leaves its sums exactly as they were; the warp leaves the chunk once all of its
        // pixels have stopped
        if (__ballot_sync(kFull, on0 || on1) == 0u) {
          if (__all_sync(kFull, done0 && done1)) break;
          continue;
        }
        const float4 q3 = sb.q3[j];
        const float2 E0 = lo_hi(q3, false), E1 = lo_hi(q3, true), E2 = lo_hi(sb.q4[j], false);
        const float2 alpha = make_float2(on0 ? fminf(amax, fast_exp2(e.x)) : 0.f, on1 ? fminf(amax, fast_exp2(e.y)) : 0.f);
        const uint32_t pos = base + j - range.x;
        bool c0, c1;  // composited (the overdraw count)
        if constexpr (KIND == NGS_MODEL_QUAD) {
          const float2 ptr = __fmul2_rn(alpha, __ffma2_rn(c2, tau, one));
          const float2 pt = make_float2(fmaxf(ptr.x, 0.f), fmaxf(ptr.y, 0.f));
          const float2 Sn = __fadd2_rn(S, pt);
          const bool s0 = on0 && Sn.x >= 1.0f, s1 = on1 && Sn.y >= 1.0f;  // the saturating splat k
          const float2 oms = __ffma2_rn(S, neg, one);                     // pbar_k = 1 - S (Eq. nexp_p)
          const float2 wc = make_float2(s0 ? oms.x : pt.x, s1 ? oms.y : pt.y);
          const float2 wa = make_float2(s0 ? 0.f : alpha.x, s1 ? 0.f : alpha.y);
          C0 = __ffma2_rn(E0, wc, C0);
          C1 = __ffma2_rn(E1, wc, C1);
          C2 = __ffma2_rn(E2, wc, C2);
          A0 = __ffma2_rn(E0, wa, A0);
          A1 = __ffma2_rn(E1, wa, A1);
          A2 = __ffma2_rn(E2, wa, A2);
          S = make_float2(s0 ? S.x : Sn.x, s1 ? S.y : Sn.y);
          tau = __fadd2_rn(tau, wa);
          if (s0) {
            Ek[0][0] = E0.x, Ek[0][1] = E1.x, Ek[0][2] = E2.x;
            sat0 = done0 = true;
            stop0 = pos + 1;
          }
          if (s1) {
            Ek[1][0] = E0.y, Ek[1][1] = E1.y, Ek[1][2] = E2.y;
            sat1 = done1 = true;
            stop1 = pos + 1;
          }
          c0 = on0;
          c1 = on1;
        } else {
          // stop before the splat that would take T below t_eps
          const float2 testT = __fmul2_rn(T, __ffma2_rn(alpha, neg, one));
          const bool st0 = on0 && testT.x < rp.t_eps, st1 = on1 && testT.y < rp.t_eps;
          if (st0) {
            done0 = true;
            stop0 = pos;
          }
          if (st1) {
            done1 = true;
            stop1 = pos;
          }
          c0 = on0 && !st0;
          c1 = on1 && !st1;
          const float2 w = __fmul2_rn(make_float2(c0 ? alpha.x : 0.f, c1 ? alpha.y : 0.f), T);
          C0 = __ffma2_rn(E0, w, C0);
          C1 = __ffma2_rn(E1, w, C1);
          C2 = __ffma2_rn(E2, w, C2);
          T = make_float2(c0 ? testT.x : T.x, c1 ? testT.y : T.y);
        }
        od0 += c0;
        od1 += c1;
        if (rp.max_splats > 0) {
          if (c0 && !done0 && od0 == rp.max_splats) {
            done0 = true;
            stop0 = pos + 1;
          }
          if (c1 && !done1 && od1 == rp.max_splats) {
            done1 = true;
            stop1 = pos + 1;
          }
        }
      }
    }
  }
  const size_t pbase = view_pix_base(rp, views, tv.view);
  float* const out_image = view_image(rp, views, tv.view, image);
  int32_t* const out_overdraw = view_overdraw(rp, views, tv.view, overdraw);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    if (!(k ? in1 : in0)) continue;
    const size_t lpix = (size_t)(y + 4 * k) * W + x;  // pixel within the view
    const size_t pix = pbase + lpix;                  // packed pixel of the replay state
    const float c0v = k ? C0.y : C0.x, c1v = k ? C1.y : C1.x, c2v = k ? C2.y : C2.x;
    const bool sat = k ? sat1 : sat0;
    const float Tend = KIND == NGS_MODEL_EXP ? (k ? T.y : T.x) : (sat ? 0.f : 1.f - (k ? S.y : S.x));
    const float L0 = c0v + rp.bg[0] * Tend, L1 = c1v + rp.bg[1] * Tend, L2 = c2v + rp.bg[2] * Tend;
    out_image[3 * lpix] = L0;
    out_image[3 * lpix + 1] = L1;
    out_image[3 * lpix + 2] = L2;
    if (out_overdraw) out_overdraw[lpix] = k ? od1 : od0;
    const uint32_t nbits = (k ? stop1 : stop0) | (sat ? 0x80000000u : 0u);
    if constexpr (KIND == NGS_MODEL_QUAD) {
      state[2 * pix] = make_float4(__uint_as_float(nbits), Ek[k][0], Ek[k][1], Ek[k][2]);
      state[2 * pix + 1] = make_float4(k ? A0.y : A0.x, k ? A1.y : A1.x, k ? A2.y : A2.x, k ? tau.y : tau.x);
    } else {
      state[2 * pix] = make_float4(__uint_as_float(nbits), L0, L1, L2);
      state[2 * pix + 1] = make_float4(Tend, 0.f, 0.f, 0.f);
    }
  }
}

// The packed forward pays where pixels walk long lists: always for the exponential model; for the quadratic
// models (rays saturate after ~8 splats, and a thread runs until the later of its two pixels stops) only on
// tiles of 256 pixels or more (measured on GB300 at 500k / 1080p: exponential 8x8 forward -10 %,
// quadratic 16x16 -1 %, quadratic 8x8 +3 % to +30 %).
template <int TW, int TH, int KIND, int CH>
constexpr bool kPairFwd = kPairForm<KIND, CH> && (KIND == NGS_MODEL_EXP || TW * TH >= 256);
template <int TW, int TH, int KIND, int CH>
constexpr int kFwdThreads = TW * TH / (kPairFwd<TW, TH, KIND, CH> ? 2 : 1);
// The packed quadratic forward on 16x16 tiles: nine CTAs of 128 threads per SM (at most 56 registers)
// instead of the eight its 64 registers would allow.
template <int TW, int TH, int KIND, int CH>
constexpr int kFwdMinBlocks = (kPairFwd<TW, TH, KIND, CH> && KIND == NGS_MODEL_QUAD && TW * TH == 256) ? 9 : 1;

template <int TW, int TH, int KIND, int CH, bool PERSIST>
__global__ void __launch_bounds__(kFwdThreads<TW, TH, KIND, CH>, kFwdMinBlocks<TW, TH, KIND, CH>)
    composite_forward_kernel(const float4* __restrict__ rec,
                                                                   const uint32_t* __restrict__ ids,
                                                                   const uint2* __restrict__ ranges, RenderParams rp,
                                                                   const ViewParams* __restrict__ views,
                                                                   float* __restrict__ image,
                                                                   int32_t* __restrict__ overdraw,
                                                                   float4* __restrict__ state,
                                                                   const uint32_t* __restrict__ work,
                                                                   uint32_t* counter) {
  pdl_wait();
  using Buf = std::conditional_t<kPairFwd<TW, TH, KIND, CH>, PairStageBuf<CH>, StageBuf<CH>>;
  __shared__ Buf sb;
  auto one_tile = [&](uint32_t tile) {
    if constexpr (kPairFwd<TW, TH, KIND, CH>)
      forward_tile_pairs<TW, TH, KIND, CH>(rec, ids, ranges, rp, views, image, overdraw, state, tile, sb);
    else
      forward_tile<TW, TH, KIND, CH>(rec, ids, ranges, rp, views, image, overdraw, state, tile, sb);
  };
  if constexpr (PERSIST) {
    __shared__ uint32_t s_next;
    for (;;) {
      const uint32_t tile = next_tile(work, counter, rp.n_tiles, &s_next);
      if (tile >= rp.n_tiles) break;
      one_tile(tile);
    }
  } else {
    one_tile(blockIdx.x);
  }
}

// ---- backward (path replay) --------------------------------------------------------------------------

struct BwdPixel {
  float px, py;
  uint32_t last;        // replay entries [range.x, last)
  float g0, g1, g2;
  float gEk, gTh, gL0;  // quadratic: g.E_k, g.Theta; exponential: g.L0; Vicini: both lists' (gEk, gL0)
  float S, tau, T, gacc;
  float P, gB, gBi;     // blended: prod (1 - alpha), g.B and its running prefix
  bool sat, stop_e;     // Vicini: the linear list saturated / the exponential list stopped
};

// Sum nine per-lane values over the warp and add the totals to dst[0..8] with one atomic instruction.
// Values 0..7 go through a transposing butterfly: at each of three steps a lane keeps half of the values
// it carries and sends the other half to its partner, so after xor 16, 8, 4 a lane carries one of them,
// summed over 8 lanes; value 8 is summed over the same lanes by a plain tree. The last two steps (xor 2,
// 1) carry both, half of the lanes each, so that lane l ends with the warp total of value ((l >> 2) & 7)
// when l % 4 == 0, and lane 2 with that of value 8: 12 shuffles instead of 45 for nine plain trees.
__device__ __forceinline__ void warp_reduce9_add(const float (&v)[9], float* dst, int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  float w[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    float send = b4 ? v[p] : v[p + 4];
    float keep = b4 ? v[p + 4] : v[p];
    w[p] = keep + __shfl_xor_sync(kFull, send, 16);
  }
  float x[2];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    float send = b3 ? w[p] : w[p + 2];
    float keep = b3 ? w[p + 2] : w[p];
    x[p] = keep + __shfl_xor_sync(kFull, send, 8);
  }
  float send = b2 ? x[0] : x[1];
  float y = (b2 ? x[1] : x[0]) + __shfl_xor_sync(kFull, send, 4);
  // the ninth value over lane bits 4..2, then both over bits 1 and 0 in one transposing step: lanes with
  // bit 1 clear carry y, lanes with it set carry e
  float e = v[8];
  e += __shfl_xor_sync(kFull, e, 16);
  e += __shfl_xor_sync(kFull, e, 8);
  e += __shfl_xor_sync(kFull, e, 4);
  const bool b1 = lane & 2;
  float z = (b1 ? e : y) + __shfl_xor_sync(kFull, b1 ? y : e, 2);
  z += __shfl_xor_sync(kFull, z, 1);
  if ((lane & 3) == 0)
    atomicAdd(dst + ((lane >> 2) & 7), z);  // value (lane >> 2) & 7, summed over the warp
  else if ((lane & 3) == 2 && lane < 4)
    atomicAdd(dst + 8, z);                  // the ninth, summed over the warp
}

// One list entry for one pixel of the replay: adds the pixel's contributions to the per-splat sums that
// do not involve dx (v[1], v[4..8]; the caller forms the dx moments once for the column) and returns
// whether the splat was composited at this pixel.
template <int KIND>
__device__ __forceinline__ bool bwd_step(BwdPixel& p, float dx, float adx, float4 r0, float4 r1, const float& e2,
                                         uint32_t pos, const RenderParams& rp, float (&v)[9]) {
  if (pos >= p.last) return false;
  float dy;
  float e = splat_log2_alpha_col(dx, adx, p.py, r0, r1, dy);
  if (e < rp.log2_alpha_min) return false;
  float raw = fast_exp2(e);
  float alpha = fminf(rp.alpha_max, raw);
  float E0 = r1.z, E1 = r1.w, E2 = e2;
  float gE = fmaf(p.g2, E2, fmaf(p.g1, E1, p.g0 * E0));  // g.E_i
  float dLda, wE;
  if constexpr (KIND == NGS_MODEL_BLEND) {
    // L0 = sum_{i<k} DeltaE_i alpha_i (1 - g + g P_i) + E_k; with B = sum_{l<k} DeltaE_l alpha_l P_l and its
    // prefix B_i = sum_{l<=i}: dL0/dalpha_i = DeltaE_i (1 - g + g P_i) - g (B - B_i) / (1 - alpha_i)
    const float pt = blend_slope(alpha, rp.c, rp.c1, p.P);
    const float Sn = __fadd_rn(p.S, pt);
    if (Sn >= 1.0f) {
      wE = 1.0f - p.S;
      dLda = 0.f;
    } else {
      const float gd = gE - p.gEk;
      p.gBi = fmaf(gd, __fmul_rn(alpha, p.P), p.gBi);
      dLda = fmaf(gd, __fmaf_rn(rp.c, p.P, rp.c1), -rp.c * (p.gB - p.gBi) * fast_rcp(1.0f - alpha));
      wE = pt;
      p.S = Sn;
      p.P = __fmul_rn(p.P, __fsub_rn(1.0f, alpha));
    }
  } else if constexpr (KIND == NGS_MODEL_VICINI) {
    // (1 - g) x the linear list's adjoint + g x the exponential list's, each up to its own stop
    float pe = 0.f, dexp = 0.f;
    if (!p.stop_e) {
      const float testT = __fmul_rn(p.T, __fsub_rn(1.0f, alpha));
      if (testT < rp.t_eps) {
        p.stop_e = true;
      } else {
        pe = alpha * p.T;
        p.gacc = fmaf(gE, pe, p.gacc);
        dexp = fmaf(p.T, gE, -fast_rcp(1.0f - alpha) * (p.gL0 - p.gacc));
        p.T = testT;
      }
    }
    float pl = 0.f, dlin = 0.f;
    if (!p.sat) {
      const float Sn = __fadd_rn(p.S, alpha);
      if (Sn >= 1.0f) {
        pl = 1.0f - p.S;
        p.S = 1.0f;
        p.sat = true;
      } else {
        pl = alpha;
        p.S = Sn;
        dlin = gE - p.gEk;
      }
    }
    dLda = fmaf(rp.c1, dlin, rp.c * dexp);
    wE = fmaf(rp.c1, pl, rp.c * pe);
  } else if constexpr (KIND == NGS_MODEL_QUAD) {
    float pt = quad_slope(alpha, rp.c, p.tau);
    float Sn = __fadd_rn(p.S, pt);
    if (Sn >= 1.0f) {  // the saturating splat k: pbar_k = 1 - S, no dependence on alpha_k
      wE = 1.0f - p.S;
      dLda = 0.f;
    } else {
      // g.dL0/dalpha_i = g.DeltaE_i (1 + c taubar_i) + c g.Theta_i, Theta_i = Theta_{i-1} - DeltaE_i alpha_i
      float gd = gE - p.gEk;
      p.gTh = fmaf(-gd, alpha, p.gTh);
      dLda = fmaf(gd, fmaf(rp.c, p.tau, 1.0f), rp.c * p.gTh);
      wE = pt;
      p.S = Sn;
      p.tau = __fadd_rn(p.tau, alpha);
    }
  } else {
    // g.dL0/dalpha_i = T_i g.E_i - (g.L0 - g.sum_{j<=i} E_j pbar_j) / (1 - alpha_i)
    wE = alpha * p.T;
    p.gacc = fmaf(gE, wE, p.gacc);
    dLda = fmaf(p.T, gE, -fast_rcp(1.0f - alpha) * (p.gL0 - p.gacc));
    p.T = __fmul_rn(p.T, __fsub_rn(1.0f, alpha));
  }
  // alpha = 2^e with e = L + dx (A' dx + B' dy) + C' dy^2, unless clamped at alpha_max. With
  // w = dL/de, de/dA' = dx^2, de/dB' = dx dy, de/dC' = dy^2, de/dL = 1 and de/du = -(2A' dx + B' dy),
  // de/dv = -(B' dx + 2C' dy): the per-splat sums of w, w dx, w dy, w dx^2, w dx dy, w dy^2 carry
  // everything; the projection backward applies the per-splat A', B', C' (and ln 2) once.
  float wgt = raw >= rp.alpha_max ? 0.f : dLda * alpha;  // dL/de / ln 2
  float wdy = wgt * dy;
  v[1] += wdy;
  v[4] = fmaf(wdy, dy, v[4]);
  v[5] += wgt;
  v[6] = fmaf(p.g0, wE, v[6]);
  v[7] = fmaf(p.g1, wE, v[7]);
  v[8] = fmaf(p.g2, wE, v[8]);
  return true;
}

// ---- backward, packed form (exponential and quadratic) -----------------------------------------------
//
// The thread's two pixels (x, y) and (x, y + 4) step through each list entry together in FP32x2
// instructions (add / mul / fma .f32x2, one instruction for both pixels). Each lane rounds exactly like
// the scalar forward, so alpha and every compositing decision are bit-identical. A pixel that does not
// composite the entry (past its stop, or alpha < alpha_min) gets alpha = 0, which leaves its running sums
// exactly as they were and contributes zero.

// Both pixels' replay state, lane 0 = pixel (x, y), lane 1 = pixel (x, y + 4).
struct BwdPair {
  float2 px, py;
  uint32_t last0, last1;  // replay entries [range.x, last)
  float2 g0, g1, g2;
  float2 T, gacc, gL0;    // exponential: T_i, g.sum_{j<i} E_j pbar_j, g.L0
  float2 S, tau, nEk, nTh;  // quadratic: S, taubar, -g.E_k, -g.Theta
};

// The quadratic form of an entry at both pixels (as splat_log2_alpha_col computes it per pixel): e = log2
// of aleph K, dx (px - u, equal in both lanes: one column) and dy.
__device__ __forceinline__ float2 pair_log2_alpha(const BwdPair& p, float4 q0, float4 q1, float4 q2, float2& dx,
                                                  float2& dy) {
  dx = __fadd2_rn(p.px, lo_hi(q0, false));
  const float2 adx = __fmul2_rn(lo_hi(q1, false), dx);
  dy = __fadd2_rn(p.py, lo_hi(q0, true));
  const float2 t = __ffma2_rn(lo_hi(q1, true), dy, adx);
  const float2 cdd = __fmul2_rn(__fmul2_rn(lo_hi(q2, false), dy), dy);
  return __fadd2_rn(lo_hi(q2, true), __ffma2_rn(dx, t, cdd));
}

// One list entry for both pixels, given the quadratic form (e, dx, dy) and which pixels composite it
// (on0 / on1: not past their stop, alpha >= alpha_min): adds their contributions to v (the 9 per-splat
// sums, the dx moments included). A pixel that does not composite it gets alpha = 0, which leaves its
// running sums exactly as they were and adds nothing, so the warp runs the step whenever any lane is on.
template <int KIND>
__device__ __forceinline__ void bwd_pair_step(BwdPair& p, float2 e, float2 dx, float2 dy, float4 q3, float4 q4,
                                              bool on0, bool on1, const RenderParams& rp, float (&v)[9]) {
  const float2 one = make_float2(1.f, 1.f), neg = make_float2(-1.f, -1.f);
  const float raw0 = fast_exp2(e.x), raw1 = fast_exp2(e.y);
  const float2 alpha = make_float2(on0 ? fminf(rp.alpha_max, raw0) : 0.f, on1 ? fminf(rp.alpha_max, raw1) : 0.f);
  // w = dL/de: zero where alpha is clamped at alpha_max (it no longer depends on e) or not composited
  bool live0 = on0 && raw0 < rp.alpha_max, live1 = on1 && raw1 < rp.alpha_max;
  const float2 gE =
      __ffma2_rn(p.g2, lo_hi(q4, false), __ffma2_rn(p.g1, lo_hi(q3, true), __fmul2_rn(p.g0, lo_hi(q3, false))));
  float2 dLda, wE;
  if constexpr (KIND == NGS_MODEL_QUAD) {
    const float2 ct = __ffma2_rn(make_float2(rp.c, rp.c), p.tau, one);  // 1 + c taubar_i
    const float2 ptr = __fmul2_rn(alpha, ct);
    const float2 pt = make_float2(fmaxf(ptr.x, 0.f), fmaxf(ptr.y, 0.f));
    const float2 Sn = __fadd2_rn(p.S, pt);
    const bool sat0 = Sn.x >= 1.0f, sat1 = Sn.y >= 1.0f;  // the saturating splat k: pbar_k = 1 - S
    const float2 oms = __ffma2_rn(p.S, neg, one);
    wE = make_float2(sat0 ? oms.x : pt.x, sat1 ? oms.y : pt.y);
    live0 = live0 && !sat0;
    live1 = live1 && !sat1;
    // -g.Theta_i = -g.Theta_{i-1} + g.DeltaE_i alpha_i; dL0/dalpha_i = g.DeltaE_i (1 + c taubar_i) + c g.Theta_i
    const float2 gd = __fadd2_rn(gE, p.nEk);
    p.nTh = __ffma2_rn(gd, alpha, p.nTh);
    dLda = __ffma2_rn(gd, ct, __fmul2_rn(make_float2(-rp.c, -rp.c), p.nTh));
    p.S = make_float2(sat0 ? p.S.x : Sn.x, sat1 ? p.S.y : Sn.y);  // S stays below 1 for later entries
    p.tau = __fadd2_rn(p.tau, alpha);
  } else {
    // dL0/dalpha_i = T_i g.E_i - (g.L0 - g.sum_{j<=i} E_j pbar_j) / (1 - alpha_i)
    wE = __fmul2_rn(alpha, p.T);
    p.gacc = __ffma2_rn(gE, wE, p.gacc);
    const float2 oma = __ffma2_rn(alpha, neg, one);
    const float2 rcp = make_float2(fast_rcp(oma.x), fast_rcp(oma.y));
    dLda = __ffma2_rn(p.T, gE, __fmul2_rn(rcp, __ffma2_rn(p.gL0, neg, p.gacc)));
    p.T = __fmul2_rn(p.T, oma);
  }
  const float2 wgt = __fmul2_rn(dLda, make_float2(live0 ? alpha.x : 0.f, live1 ? alpha.y : 0.f));
  const float2 wdy = __fmul2_rn(wgt, dy);
  const float2 wdyy = __fmul2_rn(wdy, dy);
  const float2 c0 = __fmul2_rn(p.g0, wE), c1 = __fmul2_rn(p.g1, wE), c2 = __fmul2_rn(p.g2, wE);
  v[5] = wgt.x + wgt.y;
  v[1] = wdy.x + wdy.y;
  v[4] = wdyy.x + wdyy.y;
  v[0] = dx.x * v[5];
  v[2] = dx.x * v[0];
  v[3] = dx.x * v[1];
  v[6] = c0.x + c0.y;
  v[7] = c1.x + c1.y;
  v[8] = c2.x + c2.y;
}

template <int TW, int TH, int KIND, int CH>
__device__ __forceinline__ void backward_tile_pairs(const float4* __restrict__ rec, const uint32_t* __restrict__ ids,
                                                    const uint2* __restrict__ ranges, const RenderParams& rp,
                                                    const ViewParams* __restrict__ views,
                                                    const float* __restrict__ dl_dimage,
                                                    const float4* __restrict__ state, float4* __restrict__ grad2d,
                                                    uint32_t tile, PairStageBuf<CH>& sb) {
  using G = TileGeom<TW, TH, kBwdPix>;
  constexpr int B = G::kThreads;
  const TileView tv = tile_view(rp, views, (uint32_t)tile);
  const int W = tv.W, H = tv.H;
  const size_t pix_base = view_pix_base(rp, views, tv.view);
  const int tx = tv.local % tv.tiles_x, ty = tv.local / tv.tiles_x;
  const int tid = threadIdx.x, lane = tid & 31;
  const uint2 range = ranges[tile];
  BwdPair p;
  float px[2], py[2], g[2][3], gEk[2], gThe[2], gL0[2];
  uint32_t last[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    int x, y;
    G::pixel(tid, k, tx * TW, ty * TH, x, y);
    px[k] = (float)x + 0.5f;
    py[k] = (float)y + 0.5f;
    last[k] = range.x;
    g[k][0] = g[k][1] = g[k][2] = 0.f;
    gEk[k] = gThe[k] = gL0[k] = 0.f;
    if (x < W && y < H) {
      const size_t pix = pix_base + (size_t)y * W + x;
      const float4 s0 = state[2 * pix], s1 = state[2 * pix + 1];
      last[k] = range.x + (__float_as_uint(s0.x) & 0x7FFFFFFFu);
      g[k][0] = dl_dimage[3 * pix];
      g[k][1] = dl_dimage[3 * pix + 1];
      g[k][2] = dl_dimage[3 * pix + 2];
      if constexpr (KIND == NGS_MODEL_QUAD) {
        gEk[k] = g[k][0] * s0.y + g[k][1] * s0.z + g[k][2] * s0.w;
        // Theta_{-1} = A - E_k taubar_k
        gThe[k] = g[k][0] * (s1.x - s0.y * s1.w) + g[k][1] * (s1.y - s0.z * s1.w) + g[k][2] * (s1.z - s0.w * s1.w);
      } else {
        gL0[k] = g[k][0] * s0.y + g[k][1] * s0.z + g[k][2] * s0.w;
      }
      if (g[k][0] == 0.f && g[k][1] == 0.f && g[k][2] == 0.f) last[k] = range.x;
    }
  }
  p.px = make_float2(px[0], px[0]);  // one column: px[1] == px[0]
  p.py = make_float2(py[0], py[1]);
  p.last0 = last[0];
  p.last1 = last[1];
  p.g0 = make_float2(g[0][0], g[1][0]);
  p.g1 = make_float2(g[0][1], g[1][1]);
  p.g2 = make_float2(g[0][2], g[1][2]);
  p.T = make_float2(1.f, 1.f);
  p.gacc = make_float2(0.f, 0.f);
  p.gL0 = make_float2(gL0[0], gL0[1]);
  p.S = p.tau = make_float2(0.f, 0.f);
  p.nEk = make_float2(-gEk[0], -gEk[1]);
  p.nTh = make_float2(-gThe[0], -gThe[1]);
  const uint32_t my_last = max(p.last0, p.last1);
  const uint32_t warp_last = __reduce_max_sync(kFull, my_last);
  for (uint32_t base = range.x; base < range.y; base += CH) {
    if (__syncthreads_count(base >= my_last) == B) break;
    stage_chunk_pairs<B, CH>(rec, ids, rp, base, range.y, sb);
    __syncthreads();
    if (base < warp_last) {
      const int cnt = (int)(min(warp_last, min(base + (uint32_t)CH, range.y)) - base);
      for (int j = 0; j < cnt; ++j) {
        float2 dx, dy;
        const float2 e = pair_log2_alpha(p, sb.q0[j], sb.q1[j], sb.q2[j], dx, dy);
        const uint32_t pos = base + j;
        const bool on0 = pos < p.last0 && e.x >= rp.log2_alpha_min;
        const bool on1 = pos < p.last1 && e.y >= rp.log2_alpha_min;
        const bool on = on0 || on1;
        const uint32_t mask = __ballot_sync(kFull, on);
        if (mask) {  // warp-uniform: the step is exact for the lanes that are off
          float v[9];
          const float4 q4 = sb.q4[j];
          bwd_pair_step<KIND>(p, e, dx, dy, sb.q3[j], q4, on0, on1, rp, v);
          float4* dst = grad2d + 3 * (size_t)__float_as_uint(q4.z);
          if (__popc(mask) <= kDirectLanes) {
            if (on) {
              atomicAdd(dst, make_float4(v[0], v[1], v[2], v[3]));
              atomicAdd(dst + 1, make_float4(v[4], v[5], v[6], v[7]));
              atomicAdd(reinterpret_cast<float*>(dst + 2), v[8]);
            }
          } else {
            if (!on) {
#pragma unroll
              for (int k = 0; k < 9; ++k) v[k] = 0.f;
            }
            warp_reduce9_add(v, reinterpret_cast<float*>(dst), lane);
          }
        }
      }
    }
  }
}

template <int TW, int TH, int KIND, int CH>
__device__ __forceinline__ void backward_tile(const float4* __restrict__ rec, const uint32_t* __restrict__ ids,
                                              const uint2* __restrict__ ranges, const RenderParams& rp,
                                              const ViewParams* __restrict__ views,
                                              const float* __restrict__ dl_dimage, const float4* __restrict__ state,
                                              float4* __restrict__ grad2d, uint32_t tile, StageBuf<CH>& sb,
                                              uint32_t* s_id) {
  using G = TileGeom<TW, TH, kBwdPix>;
  constexpr int B = G::kThreads;
  static_assert(kBwdPix == 2, "the replay below is written for two pixels per thread");
  const TileView tv = tile_view(rp, views, (uint32_t)tile);
  const int W = tv.W, H = tv.H;
  const size_t pix_base = view_pix_base(rp, views, tv.view);
  const int tx = tv.local % tv.tiles_x, ty = tv.local / tv.tiles_x;
  const int tid = threadIdx.x, lane = tid & 31;
  const uint2 range = ranges[tile];
  BwdPixel p[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    int x, y;
    G::pixel(tid, k, tx * TW, ty * TH, x, y);
    BwdPixel& q = p[k];
    q.px = (float)x + 0.5f;
    q.py = (float)y + 0.5f;
    q.last = range.x;
    q.g0 = q.g1 = q.g2 = 0.f;
    // everything the adjoint needs is a dot product with g: quadratic keeps g.E_k and g.Theta,
    // exponential keeps g.L0 and the running g.sum_{j<=i} E_j pbar_j
    q.gEk = q.gTh = q.gL0 = 0.f;
    q.S = q.tau = q.gacc = 0.f;
    q.T = 1.f;
    q.P = 1.f;
    q.gB = q.gBi = 0.f;
    q.sat = q.stop_e = false;
    if (x < W && y < H) {
      size_t pix = pix_base + (size_t)y * W + x;
      float4 s0 = state[2 * pix], s1 = state[2 * pix + 1];
      q.last = range.x + (__float_as_uint(s0.x) & 0x7FFFFFFFu);
      q.g0 = dl_dimage[3 * pix];
      q.g1 = dl_dimage[3 * pix + 1];
      q.g2 = dl_dimage[3 * pix + 2];
      if constexpr (KIND == NGS_MODEL_QUAD) {
        q.gEk = q.g0 * s0.y + q.g1 * s0.z + q.g2 * s0.w;
        // Theta_{-1} = A - E_k taubar_k
        q.gTh = q.g0 * (s1.x - s0.y * s1.w) + q.g1 * (s1.y - s0.z * s1.w) + q.g2 * (s1.z - s0.w * s1.w);
      } else if constexpr (KIND == NGS_MODEL_BLEND) {
        q.gEk = q.g0 * s0.y + q.g1 * s0.z + q.g2 * s0.w;
        // B = sum_{l<k} E_l alpha_l P_l - E_k sum_{l<k} alpha_l P_l
        q.gB = q.g0 * s1.x + q.g1 * s1.y + q.g2 * s1.z - q.gEk * s1.w;
      } else if constexpr (KIND == NGS_MODEL_VICINI) {
        q.gEk = q.g0 * s0.y + q.g1 * s0.z + q.g2 * s0.w;  // E_k of the linear list
        q.gL0 = q.g0 * s1.x + q.g1 * s1.y + q.g2 * s1.z;  // L0 of the exponential list
      } else {
        q.gL0 = q.g0 * s0.y + q.g1 * s0.z + q.g2 * s0.w;
      }
      if (q.g0 == 0.f && q.g1 == 0.f && q.g2 == 0.f) q.last = range.x;
    }
  }
  // the warp walks entries up to the largest stop of its pixels
  const uint32_t warp_last = __reduce_max_sync(kFull, max(p[0].last, p[1].last));
  for (uint32_t base = range.x; base < range.y; base += CH) {
    const bool done = base >= max(p[0].last, p[1].last);
    if (__syncthreads_count(done) == B) break;
    stage_chunk<B, CH>(rec, ids, rp, base, range.y, sb, s_id);
    __syncthreads();
    if (base < warp_last) {
      const int cnt = (int)(min(warp_last, min(base + (uint32_t)CH, range.y)) - base);
      for (int j = 0; j < cnt; ++j) {
        const uint32_t pos = base + j;
        const float4 r0 = sb.r0[j], r1 = sb.r1[j];
        // both pixels of the thread lie in one column: dx and A' dx are shared, and the dx moments
        // follow from the others (sum w dx = dx sum w, sum w dx^2 = dx^2 sum w, sum w dx dy = dx sum w dy)
        const float dx = __fsub_rn(p[0].px, r0.x), adx = __fmul_rn(r0.z, dx);
        float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        bool on = bwd_step<KIND>(p[0], dx, adx, r0, r1, sb.e2[j], pos, rp, v);
        on |= bwd_step<KIND>(p[1], dx, adx, r0, r1, sb.e2[j], pos, rp, v);
        v[0] = dx * v[5];
        v[2] = dx * v[0];
        v[3] = dx * v[1];
        const uint32_t mask = __ballot_sync(kFull, on);
        if (mask) {
          float4* dst = grad2d + 3 * (size_t)s_id[j];
          // up to kDirectLanes lanes add their values with their own vector atomics (3 instructions) rather
          // than through the warp reduction (about 70); a full warp hitting one splat reduces first, since
          // 32 atomics on one address serialise
          if (__popc(mask) <= kDirectLanes) {
            if (on) {
              atomicAdd(dst, make_float4(v[0], v[1], v[2], v[3]));
              atomicAdd(dst + 1, make_float4(v[4], v[5], v[6], v[7]));
              atomicAdd(reinterpret_cast<float*>(dst + 2), v[8]);
            }
          } else {
            warp_reduce9_add(v, reinterpret_cast<float*>(dst), lane);
          }
        }
      }
    }
  }
}

template <int TW, int TH, int KIND, int CH, bool PERSIST>
__global__ void __launch_bounds__(TW* TH / kBwdPix) composite_backward_kernel(const float4* __restrict__ rec,
                                                                        const uint32_t* __restrict__ ids,
                                                                        const uint2* __restrict__ ranges,
                                                                        RenderParams rp,
                                                                        const ViewParams* __restrict__ views,
                                                                        const float* __restrict__ dl_dimage,
                                                                        const float4* __restrict__ state,
                                                                        float4* __restrict__ grad2d,
                                                                        const uint32_t* __restrict__ work,
                                                                        uint32_t* counter) {
  pdl_wait();
  using Buf = std::conditional_t<kPairForm<KIND, CH>, PairStageBuf<CH>, StageBuf<CH>>;
  __shared__ Buf sb;
  __shared__ uint32_t s_id[kPairForm<KIND, CH> ? 1 : CH];  // the packed form carries the index in its q4
  auto one_tile = [&](uint32_t tile) {
    if constexpr (kPairForm<KIND, CH>)
      backward_tile_pairs<TW, TH, KIND, CH>(rec, ids, ranges, rp, views, dl_dimage, state, grad2d, tile, sb);
    else
      backward_tile<TW, TH, KIND, CH>(rec, ids, ranges, rp, views, dl_dimage, state, grad2d, tile, sb, s_id);
  };
  if constexpr (PERSIST) {
    __shared__ uint32_t s_next;
    for (;;) {
      const uint32_t tile = next_tile(work, counter, rp.n_tiles, &s_next);
      if (tile >= rp.n_tiles) break;
      one_tile(tile);
    }
  } else {
    one_tile(blockIdx.x);
  }
}

// Launch configuration of a composite launch: chunk factor (records staged per round = tile pixels x
// {1/2, 1, 2}) and schedule (one CTA per tile, or persistent CTAs over the work list).
struct Launch {
  int chunk_code;                   // 0: half, 1: equal, 2: double the tile's pixel count
  const uint32_t* work;             // persistent schedule: tile order (null: identity)
  uint32_t* counter;                // persistent schedule: zeroed work counter (null: one CTA per tile)
  int num_sms;
};

// One CTA per tile, or one wave of persistent CTAs (SM count x resident CTAs per SM).
template <typename Kernel>
static unsigned grid_for(Kernel k, int threads, const Launch& L, uint32_t n_tiles) {
  if (!L.counter) return n_tiles;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
  return (unsigned)std::min<uint64_t>((uint64_t)per_sm * (uint64_t)L.num_sms, n_tiles);
}

template <int TW, int TH, int KIND, int CH>
void forward_launch(const float4* rec, const uint32_t* ids, const uint2* ranges, const RenderParams& rp,
                    const ViewParams* views, float* image, int32_t* overdraw, float4* state, const Launch& L,
                    cudaStream_t s) {
  constexpr int threads = kFwdThreads<TW, TH, KIND, CH>;
  auto k = L.counter ? composite_forward_kernel<TW, TH, KIND, CH, true> : composite_forward_kernel<TW, TH, KIND, CH, false>;
  launch_pdl(k, grid_for(k, threads, L, rp.n_tiles), threads, 0, s, rec, ids, ranges, rp, views, image, overdraw, state,
             L.work, L.counter);
}

template <int TW, int TH, int KIND, int CH>
void backward_launch(const float4* rec, const uint32_t* ids, const uint2* ranges, const RenderParams& rp,
                     const ViewParams* views, const float* dl, const float4* state, float4* grad2d, const Launch& L,
                     cudaStream_t s) {
  constexpr int threads = TileGeom<TW, TH, kBwdPix>::kThreads;
  auto k =
      L.counter ? composite_backward_kernel<TW, TH, KIND, CH, true> : composite_backward_kernel<TW, TH, KIND, CH, false>;
  launch_pdl(k, grid_for(k, threads, L, rp.n_tiles), threads, 0, s, rec, ids, ranges, rp, views, dl, state, grad2d,
             L.work, L.counter);
}

template <int TW, int TH, int KIND>
void forward_chunk(const float4* rec, const uint32_t* ids, const uint2* ranges, const RenderParams& rp,
                   const ViewParams* views, float* image, int32_t* overdraw, float4* state, const Launch& L,
                   cudaStream_t s) {
  constexpr int P = TW * TH;
  if (L.chunk_code == 0) forward_launch<TW, TH, KIND, P / 2>(rec, ids, ranges, rp, views, image, overdraw, state, L, s);
  else if (L.chunk_code == 2) forward_launch<TW, TH, KIND, 2 * P>(rec, ids, ranges, rp, views, image, overdraw, state, L, s);
  else forward_launch<TW, TH, KIND, P>(rec, ids, ranges, rp, views, image, overdraw, state, L, s);
}

template <int TW, int TH, int KIND>
void backward_chunk(const float4* rec, const uint32_t* ids, const uint2* ranges, const RenderParams& rp,
                    const ViewParams* views, const float* dl, const float4* state, float4* grad2d, const Launch& L,
                    cudaStream_t s) {
  constexpr int P = TW * TH;
  if (L.chunk_code == 0) backward_launch<TW, TH, KIND, P / 2>(rec, ids, ranges, rp, views, dl, state, grad2d, L, s);
  else if (L.chunk_code == 2) backward_launch<TW, TH, KIND, 2 * P>(rec, ids, ranges, rp, views, dl, state, grad2d, L, s);
  else backward_launch<TW, TH, KIND, P>(rec, ids, ranges, rp, views, dl, state, grad2d, L, s);
}

template <int TW, int TH>
void forward_kind(const float4* rec, const uint32_t* ids, const uint2* ranges, const RenderParams& rp,
                  const ViewParams* views, float* image, int32_t* overdraw, float4* state, const Launch& L,
                  cudaStream_t s) {
  switch (rp.kind) {
    case NGS_MODEL_QUAD:
      forward_chunk<TW, TH, NGS_MODEL_QUAD>(rec, ids, ranges, rp, views, image, overdraw, state, L, s);
      break;
    case NGS_MODEL_BLEND:
      forward_chunk<TW, TH, NGS_MODEL_BLEND>(rec, ids, ranges, rp, views, image, overdraw, state, L, s);
      break;
    case NGS_MODEL_VICINI:
      forward_chunk<TW, TH, NGS_MODEL_VICINI>(rec, ids, ranges, rp, views, image, overdraw, state, L, s);
      break;
    default:
      forward_chunk<TW, TH, NGS_MODEL_EXP>(rec, ids, ranges, rp, views, image, overdraw, state, L, s);
  }
}

template <int TW, int TH>
void backward_kind(const float4* rec, const uint32_t* ids, const uint2* ranges, const RenderParams& rp,
                   const ViewParams* views, const float* dl, const float4* state, float4* grad2d, const Launch& L,
                   cudaStream_t s) {
  switch (rp.kind) {
    case NGS_MODEL_QUAD:
      backward_chunk<TW, TH, NGS_MODEL_QUAD>(rec, ids, ranges, rp, views, dl, state, grad2d, L, s);
      break;
    case NGS_MODEL_BLEND:
      backward_chunk<TW, TH, NGS_MODEL_BLEND>(rec, ids, ranges, rp, views, dl, state, grad2d, L, s);
      break;
    case NGS_MODEL_VICINI:
      backward_chunk<TW, TH, NGS_MODEL_VICINI>(rec, ids, ranges, rp, views, dl, state, grad2d, L, s);
      break;
    default:
      backward_chunk<TW, TH, NGS_MODEL_EXP>(rec, ids, ranges, rp, views, dl, state, grad2d, L, s);
  }
}

int chunk_code(const RenderParams& rp) {
  const int P = rp.tile_w * rp.tile_h;
  return rp.chunk == P / 2 ? 0 : rp.chunk == 2 * P ? 2 : 1;
}

}  // namespace

void launch_composite_forward(const float4* rec, const uint32_t* ids, const uint2* ranges, const RenderParams& rp,
                              const ViewParams* views, float* image, int32_t* overdraw, float4* state,
                              const uint32_t* work, uint32_t* counter, int num_sms, cudaStream_t s) {
  const Launch L{chunk_code(rp), work, counter, num_sms};
  if (rp.tile_w == 8 && rp.tile_h == 8)
    forward_kind<8, 8>(rec, ids, ranges, rp, views, image, overdraw, state, L, s);
  else if (rp.tile_w == 16 && rp.tile_h == 16)
    forward_kind<16, 16>(rec, ids, ranges, rp, views, image, overdraw, state, L, s);
  else
    forward_kind<16, 32>(rec, ids, ranges, rp, views, image, overdraw, state, L, s);
}

void launch_composite_backward(const float4* rec, const uint32_t* ids, const uint2* ranges, const RenderParams& rp,
                               const ViewParams* views, const float* dl_dimage, const float4* state, float4* grad2d,
                               const uint32_t* work, uint32_t* counter, int num_sms, cudaStream_t s) {
  const Launch L{chunk_code(rp), work, counter, num_sms};
  if (rp.tile_w == 8 && rp.tile_h == 8)
    backward_kind<8, 8>(rec, ids, ranges, rp, views, dl_dimage, state, grad2d, L, s);
  else if (rp.tile_w == 16 && rp.tile_h == 16)
    backward_kind<16, 16>(rec, ids, ranges, rp, views, dl_dimage, state, grad2d, L, s);
  else
    backward_kind<16, 32>(rec, ids, ranges, rp, views, dl_dimage, state, grad2d, L, s);
}

}  // namespace ngs
