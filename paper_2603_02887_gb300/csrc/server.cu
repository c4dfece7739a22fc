// Render server: resident scenes, continuous batching of render requests, admission by sort-buffer bytes.
//
// Workers: each is one host thread with its own CUDA stream, context and frame, so the batches of
// different workers run side by side on the device (the host synchronisation inside a render -- reading
// the pair count -- blocks only its own worker). A worker that becomes free takes the oldest pending
// request and, with it, every pending request for the same scene and transmittance model (in arrival
// order, up to max_batch_views): requests that arrived while the GPU was busy join the next batch. The
// batch is one multi-view render; each request's image is written to the caller's own buffer.
//
// Admission: the memory a render needs is known in two steps, as ngs_workspace_bytes reports it -- the
// frame's record, tile and pixel buffers and the context's scratch before the render starts, the pair
// buffers (16 bytes per pair) once the exact pair count is read back. Each step reserves its bytes against
// mem_budget and waits while they do not fit;
// the oldest batch in flight may always go on (so some batch always makes progress), and is counted as an
// over-budget admission when it had to exceed the budget to do so.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include <string.h>

#include "ngs_internal.cuh"

using namespace ngs;

namespace {

struct Pending {
  ngs_request req;
  double submit_s;
};

}  // namespace

struct ngs_server {
  ngs_server_config cfg;
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::vector<ngs_gaussians> scenes;
  std::mutex mu;
  std::condition_variable cv_work, cv_mem, cv_done;
  std::deque<Pending> queue;
  std::deque<ngs_completion> done;
  std::set<int64_t> in_flight;  // admission sequence numbers of the batches holding reservations
  int64_t next_seq = 0;
  int64_t reserved = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  ngs_server_stats stats;
  std::string err;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

struct Reservation {
  ngs_server* S;
  int64_t seq = -1;
  int64_t bytes = 0;
};

int admit(void* user, int stage, size_t bytes) {
  Reservation* r = static_cast<Reservation*>(user);
  ngs_server* S = r->S;
  std::unique_lock<std::mutex> lk(S->mu);
  if (stage == 0) r->seq = S->next_seq++;
  auto oldest = [&] { return S->in_flight.empty() || *S->in_flight.begin() >= r->seq; };
  auto fits = [&] { return S->reserved + (int64_t)bytes <= S->cfg.mem_budget; };
  S->cv_mem.wait(lk, [&] { return fits() || oldest(); });
  if (!fits()) ++S->stats.over_budget_admissions;
  if (stage == 0) S->in_flight.insert(r->seq);
  S->reserved += (int64_t)bytes;
  r->bytes += (int64_t)bytes;
  S->stats.peak_reserved_bytes = std::max(S->stats.peak_reserved_bytes, S->reserved);
  return NGS_OK;
}

void release(Reservation& r) {
  ngs_server* S = r.S;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->reserved -= r.bytes;
    if (r.seq >= 0) S->in_flight.erase(r.seq);
    r.bytes = 0;
  }
  S->cv_mem.notify_all();
}

void worker_main(ngs_server* S) {
  cudaSetDevice(S->device);
  ngs_ctx* ctx = nullptr;
  ngs_frame* f = nullptr;
  cudaStream_t st = nullptr;
  int rc0 = ngs_create(&ctx);
  if (rc0 == NGS_OK) rc0 = ngs_frame_create(ctx, &f);
  if (rc0 == NGS_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc0 = NGS_ERR_CUDA;
  if (rc0 == NGS_OK && S->cfg.graphs) ngs_set_graphs(ctx, 1);
  std::vector<Pending> batch;
  std::vector<ngs_camera> cams;
  std::vector<float*> images;
  std::vector<int32_t*> ods;
  for (;;) {
    batch.clear();
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
      if (S->queue.empty()) break;  // stopping and drained
      // the oldest request sets the scene and model; every pending request with both joins, in order
      const ngs_request& head = S->queue.front().req;
      const int32_t scene = head.scene, kind = head.model.kind;
      const float param = head.model.param;
      for (auto it = S->queue.begin(); it != S->queue.end() && (int)batch.size() < S->cfg.max_batch_views;) {
        if (it->req.scene == scene && it->req.model.kind == kind && it->req.model.param == param) {
          batch.push_back(*it);
          it = S->queue.erase(it);
        } else {
          ++it;
        }
      }
    }
    const int n = (int)batch.size();
    cams.resize(n);
    images.resize(n);
    ods.resize(n);
    for (int i = 0; i < n; ++i) {
      cams[i] = batch[i].req.camera;
      images[i] = batch[i].req.image;
      ods[i] = batch[i].req.overdraw;
    }
    const double start = S->now();
    Reservation res{S};
    int rc = rc0;
    if (rc == NGS_OK) {
      const ngs_request& r0 = batch[0].req;
      rc = render_views_out(ctx, f, &S->scenes[r0.scene], cams.data(), n, &r0.model, &S->cfg.options, images.data(),
                            ods.data(), st, admit, &res);
      if (rc == NGS_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = NGS_ERR_CUDA;
    }
    const int64_t pairs = rc == NGS_OK ? f->pairs : 0;
    release(res);
    const double end = S->now();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      if (rc != NGS_OK && S->err.empty()) S->err = ctx ? ngs_last_error(ctx) : "worker set-up failed";
      for (const Pending& p : batch) {
        ngs_completion c;
        c.tag = p.req.tag;
        c.status = rc;
        c.batch_views = n;
        c.submit_s = p.submit_s;
        c.start_s = start;
        c.done_s = end;
        c.pairs = pairs;
        S->done.push_back(c);
      }
      S->stats.completed += n;
      S->stats.batches += 1;
      S->stats.max_batch_views = std::max<int64_t>(S->stats.max_batch_views, n);
    }
    S->cv_done.notify_all();
  }
  if (st) cudaStreamDestroy(st);
  if (f) ngs_frame_destroy(f);
  if (ctx) ngs_destroy(ctx);
}

}  // namespace

extern "C" {

NGS_API void ngs_default_server_config(ngs_server_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->workers = 4;
  c->max_batch_views = 16;
  c->mem_budget = 8ll << 30;
  c->graphs = 0;  // batch shapes vary from batch to batch: replays would rarely match a capture
  ngs_default_options(&c->options);
}

NGS_API int ngs_server_create(const ngs_server_config* cfg, ngs_server** out) {
  if (!cfg || !out) return NGS_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->workers < 1 || cfg->workers > 64 || cfg->max_batch_views < 1 || cfg->max_batch_views > 4096 ||
      cfg->mem_budget < 1)
    return NGS_ERR_INVALID_ARG;
  ngs_server* S = new (std::nothrow) ngs_server();
  if (!S) return NGS_ERR_OUT_OF_MEMORY;
  S->cfg = *cfg;
  memset(&S->stats, 0, sizeof S->stats);
  S->t0 = std::chrono::steady_clock::now();
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return NGS_ERR_CUDA;
  }
  try {
    for (int i = 0; i < cfg->workers; ++i) S->workers.emplace_back(worker_main, S);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    delete S;
    return NGS_ERR_OUT_OF_MEMORY;
  }
  *out = S;
  return NGS_OK;
}

NGS_API int ngs_server_add_scene(ngs_server* S, const ngs_gaussians* g, int32_t* id) {
  if (!S || !g || !id || g->n < 0 || g->sh_degree < 0 || g->sh_degree > 3) return NGS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  S->scenes.push_back(*g);
  *id = (int32_t)S->scenes.size() - 1;
  return NGS_OK;
}

NGS_API int ngs_server_submit(ngs_server* S, const ngs_request* r) {
  if (!S || !r || !r->image) return NGS_ERR_INVALID_ARG;
  // a request that cannot render is refused here, so that it never fails a batch it would have joined
  if (check_camera(nullptr, &r->camera) != NGS_OK || check_model(nullptr, &r->model) != NGS_OK)
    return NGS_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (r->scene < 0 || r->scene >= (int32_t)S->scenes.size() || S->stop) return NGS_ERR_INVALID_ARG;
    S->queue.push_back(Pending{*r, S->now()});
    S->stats.submitted += 1;
  }
  S->cv_work.notify_one();
  return NGS_OK;
}

NGS_API int ngs_server_poll(ngs_server* S, ngs_completion* out, int32_t cap, int32_t wait_ms) {
  if (!S || (!out && cap > 0) || cap < 0) return NGS_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->done.empty() && wait_ms > 0)
    S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !S->done.empty(); });
  int n = 0;
  while (n < cap && !S->done.empty()) {
    out[n++] = S->done.front();
    S->done.pop_front();
  }
  return n;
}

NGS_API int ngs_server_get_stats(ngs_server* S, ngs_server_stats* out) {
  if (!S || !out) return NGS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->stats;
  out->pending = (int64_t)S->queue.size();
  out->reserved_bytes = S->reserved;
  out->now_s = S->now();
  return NGS_OK;
}

NGS_API const char* ngs_server_last_error(ngs_server* S) {
  if (!S) return "null server";
  std::lock_guard<std::mutex> lk(S->mu);
  return S->err.c_str();
}

NGS_API void ngs_server_destroy(ngs_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  delete S;
}

}  // extern "C"
