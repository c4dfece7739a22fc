// Autotuner over the composite's launch configuration: tile shape, records staged per round (chunk) and
// schedule. None of them changes a result (the per-tile splat lists and the per-pixel arithmetic are the
// same), so the tuner only times: one untimed render per candidate, then `reps` timed ones.
#include <algorithm>
#include <vector>

#include "ngs_internal.cuh"

using namespace ngs;

#define NGS_TRY_TUNE(x)            \
  do {                             \
    int _rc = (x);                 \
    if (_rc != NGS_OK) return _rc; \
  } while (0)

extern "C" NGS_API int ngs_autotune(ngs_ctx* ctx, ngs_frame* f, const ngs_gaussians* g, const ngs_camera* cams,
                                    int32_t n_views, const ngs_model* model, const ngs_options* base, float* images,
                                    int32_t* overdraw, const float* dl_dimage, const ngs_grads* grads, int32_t reps,
                                    int64_t flush_bytes, ngs_options* best, ngs_tune_entry* table, int32_t table_cap,
                                    void* stream) {
  if (!ctx) return NGS_ERR_INVALID_ARG;
  if (!base || !best || reps < 1 || reps > 100 || table_cap < 0 || flush_bytes < 0 || flush_bytes > (1ll << 34))
    return fail(ctx, NGS_ERR_INVALID_ARG, "autotune: null base/best, reps outside 1..100 or flush_bytes > 16 GiB");
  if (flush_bytes > 0) NGS_TRY_TUNE(ensure(ctx, ctx->flush, (size_t)flush_bytes));
  const bool with_backward = dl_dimage && grads;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(ctx, NGS_ERR_CUDA, "autotune: cudaEventCreate failed");
  }
  static const int kTiles[3][2] = {{8, 8}, {16, 16}, {16, 32}};
  int count = 0, rc = NGS_OK;
  float best_ms = 0.f;
  std::vector<float> times;
  for (const auto& t : kTiles) {
    for (int c = 0; c < 3 && rc == NGS_OK; ++c) {
      for (int sched = 0; sched < 2 && rc == NGS_OK; ++sched) {
        ngs_options o = *base;
        o.tile_w = t[0];
        o.tile_h = t[1];
        const int P = t[0] * t[1];
        o.chunk = c == 0 ? P / 2 : c == 1 ? P : 2 * P;
        o.schedule = sched;
        times.clear();
        for (int r = -1; r < reps && rc == NGS_OK; ++r) {
          if (r >= 0 && flush_bytes > 0) {
            const cudaError_t fe = cudaMemsetAsync(ctx->flush.p, r & 0xFF, (size_t)flush_bytes, s);
            if (fe != cudaSuccess) {
              rc = fail(ctx, NGS_ERR_CUDA, std::string("autotune: clearing L2: ") + cudaGetErrorString(fe));
              break;
            }
          }
          if (r >= 0) cudaEventRecord(e0, s);
          rc = render_views(ctx, f, g, cams, n_views, model, &o, images, overdraw, s);
          if (rc == NGS_OK && with_backward) rc = backward_frame(ctx, f, g, dl_dimage, grads, s);
          if (rc == NGS_OK && r >= 0) {
            float ms = 0.f;
            cudaEventRecord(e1, s);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) rc = fail(ctx, NGS_ERR_CUDA, std::string("autotune timing: ") + cudaGetErrorString(e));
            times.push_back(ms);
          }
        }
        if (rc != NGS_OK) break;
        std::sort(times.begin(), times.end());
        const float med = times[times.size() / 2];
        if (count < table_cap && table) table[count] = ngs_tune_entry{o.tile_w, o.tile_h, o.chunk, o.schedule, med};
        if (count == 0 || med < best_ms) {
          best_ms = med;
          *best = o;
        }
        ++count;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc == NGS_OK ? count : rc;
}
