// Serving loop: resident factorizations, memory-admitted builds, and
// continuous batching of right-hand sides.
//
// Each registered handle owns a worker thread, a compute stream and a copy
// stream.  The worker repeatedly takes every solve request queued for its
// handle (up to max_cols columns in total), copies their columns from the
// callers' host buffers into one device batch, runs one mixed-precision
// refined solve (rs_solve_refined) on it and copies each request's columns
// back.  Two batch buffers form a pipeline: before a batch's solve starts,
// the next batch (the requests queued by then) is taken and its columns
// copied in on the copy stream, and a finished batch's columns are copied
// back on the copy stream while the next solve runs; its requests complete
// from a host callback once that copy lands.  Requests that arrive while a
// batch is on the GPU wait for a later one, so batches form continuously.
// Workers of different handles stage and return columns concurrently but
// take turns for the solves themselves (one refined solve on the GPU at a
// time): every solve is a persistent launch sized to fill the GPU, and
// concurrent ones from several streams contend for the SMs (on the
// config-5 mix over 60 s, 17.9k right-hand sides per second concurrently
// against 21.3k taking turns).  Builds
// run on a builder thread and are admitted only while the estimated device
// memory of the resident factorizations plus the new one stays under the
// server's budget.
//
// A request's latency is the host time from submit to completion.
#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "rs_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket = 0;
  int kind = 0;              // 0 solve, 1 build
  int hid = -1;              // handle id (solve)
  const void* B = nullptr;   // host, column-major
  int64_t ldb = 0;
  void* X = nullptr;
  int64_t ldx = 0;
  int ncols = 0;
  double tol = 1e-10;
  // build
  std::vector<double> pts;
  std::vector<double> nrm, kap;   // double layer: host copies of the normals and curvatures
  int64_t n = 0;
  int dim = 2;
  rs_params params{};
  double eps = 0;
  int leaf = 0;
  // completion
  Clock::time_point t_submit, t_done;
  bool done = false;
  int status = RS_OK;
  double relres = 0;
  int its = 0;
  int result_hid = -1;       // build: id of the new handle
};

struct Worker;

struct Server {
  int max_cols = 256;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_done;
  std::map<int64_t, std::shared_ptr<Request>> reqs;
  int64_t next_ticket = 1;
  std::vector<std::unique_ptr<Worker>> workers;   // index = handle id
  // builder
  std::deque<std::shared_ptr<Request>> build_q;
  std::condition_variable cv_build;
  std::thread builder;
  bool stop = false;
  size_t resident_bytes = 0;
  // statistics
  std::vector<double> lat_ms;
  int64_t rhs_done = 0, batches = 0, batch_cols = 0;
  Clock::time_point t0 = Clock::now();
  std::mutex gpu_mu;   // held by the worker whose refined solve is on the GPU
};

struct Worker {
  Server* s = nullptr;
  rs_handle h = nullptr;
  bool owned = false;
  int id = -1;
  int64_t n = 0;
  bool cplx = false;
  cudaStream_t stream = nullptr;   // solves
  cudaStream_t cstream = nullptr;  // copies in and out
  std::deque<std::shared_ptr<Request>> q;
  std::condition_variable cv;
  std::thread th;
  // two pipeline slots: device batch buffers (n x max_cols scalars) and events
  void* db[2] = {nullptr, nullptr};
  void* dx[2] = {nullptr, nullptr};
  cudaEvent_t in_done[2] = {nullptr, nullptr};    // columns copied in
  cudaEvent_t out_done[2] = {nullptr, nullptr};   // columns copied back (slot free again)
  size_t cap = 0;

  void run();
  int take(std::vector<std::shared_ptr<Request>>& batch, int& cols, bool wait);
  int stage_in(int slot, const std::vector<std::shared_ptr<Request>>& batch);
};

// A finished batch whose columns are on their way back to the callers.
struct Finished {
  Server* s;
  std::vector<std::shared_ptr<Request>> batch;
  int rc;
  int cols;
};

size_t handle_bytes(rs_handle h) {
  rs_stats_t st;
  if (rs_stats(h, &st) != RS_OK) return 0;
  // FP64 + FP32 factors, forward blocks and solve workspaces: about 3x the FP64 factors
  return (size_t)st.factor_bytes * 3;
}

void complete(Server* s, const std::shared_ptr<Request>& r, int status) {
  r->t_done = Clock::now();
  r->status = status;
  r->done = true;
  double ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  if (status == RS_OK && r->kind == 0) {
    s->lat_ms.push_back(ms);
    s->rhs_done += r->ncols;
  }
}

// Requests for one batch (up to max_cols columns); waits for the first one
// only if `wait`.  Returns 0 when the server stops with nothing queued.
int Worker::take(std::vector<std::shared_ptr<Request>>& batch, int& cols, bool wait) {
  batch.clear();
  cols = 0;
  std::unique_lock<std::mutex> lk(s->mu);
  if (wait) cv.wait(lk, [&] { return s->stop || !q.empty(); });
  if (q.empty()) return s->stop ? 0 : 1;
  while (!q.empty() && (batch.empty() || cols + q.front()->ncols <= s->max_cols)) {
    cols += q.front()->ncols;
    batch.push_back(q.front());
    q.pop_front();
  }
  return 1;
}

// Copy a batch's columns into slot `slot` on the copy stream (after the
// slot's previous columns have gone back to their callers).
int Worker::stage_in(int slot, const std::vector<std::shared_ptr<Request>>& batch) {
  const size_t sb = cplx ? 16 : 8;
  if (cudaEventSynchronize(out_done[slot]) != cudaSuccess) {
    cudaGetLastError();
    return RS_ERR_CUDA;
  }
  size_t col = 0;
  for (auto& r : batch) {
    // contiguous columns: one plain copy (the pitched form ran at half the link's rate)
    const cudaError_t e =
        r->ldb == n ? cudaMemcpyAsync((char*)db[slot] + col * n * sb, r->B, n * sb * r->ncols, cudaMemcpyHostToDevice,
                                      cstream)
                    : cudaMemcpy2DAsync((char*)db[slot] + col * n * sb, n * sb, r->B, r->ldb * sb, n * sb, r->ncols,
                                        cudaMemcpyHostToDevice, cstream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return RS_ERR_CUDA;
    }
    col += r->ncols;
  }
  if (cudaEventRecord(in_done[slot], cstream) != cudaSuccess) {
    cudaGetLastError();
    return RS_ERR_CUDA;
  }
  return RS_OK;
}

void finish_batch(void* p) {   // host callback: no CUDA calls
  Finished* f = static_cast<Finished*>(p);
  {
    std::lock_guard<std::mutex> lk(f->s->mu);
    for (auto& r : f->batch) complete(f->s, r, f->rc);
    f->s->batches += 1;
    f->s->batch_cols += f->cols;
  }
  f->s->cv_done.notify_all();
  delete f;
}

void Worker::run() {
  const size_t sb = cplx ? 16 : 8;
  int rc0 = RS_OK;
  const size_t want = (size_t)n * s->max_cols * sb;
  for (int i = 0; i < 2 && rc0 == RS_OK; ++i) {
    if (cudaMalloc(&db[i], want) != cudaSuccess || cudaMalloc(&dx[i], want) != cudaSuccess ||
        cudaEventCreateWithFlags(&in_done[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&out_done[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(out_done[i], cstream) != cudaSuccess) {
      cudaGetLastError();
      rc0 = RS_ERR_OOM;
    }
  }
  cap = rc0 == RS_OK ? want : 0;
  std::vector<std::shared_ptr<Request>> cur, next;
  int cur_cols = 0, next_cols = 0, slot = 0;
  bool staged = false;   // cur is already in slot `slot`
  for (;;) {
    if (cur.empty()) {
      if (!take(cur, cur_cols, true)) return;
      staged = false;
    }
    int rc = rc0;
    if (rc == RS_OK && !staged) rc = stage_in(slot, cur);
    // the next batch goes in on the copy stream while this one is solved
    next.clear();
    next_cols = 0;
    bool next_staged = false;
    if (rc == RS_OK && take(next, next_cols, false) && !next.empty())
      next_staged = stage_in(slot ^ 1, next) == RS_OK;
    double tol = 1e-10;
    for (auto& r : cur) tol = std::min(tol, r->tol);
    std::vector<double> rel(cur_cols, 0.0);
    int its = 0;
    if (rc == RS_OK && cudaStreamWaitEvent(stream, in_done[slot], 0) != cudaSuccess) {
      cudaGetLastError();
      rc = RS_ERR_CUDA;
    }
    if (rc == RS_OK) {   // one solve at a time (the copies keep overlapping on the copy streams)
      std::lock_guard<std::mutex> g(s->gpu_mu);
      rc = rs_solve_refined(h, db[slot], n, cur_cols, dx[slot], n, tol, 8, &its, rel.data(), stream);
    }
    // columns back on the copy stream once the solve is done; completion from a callback
    cudaEvent_t solved;
    bool ok = cudaEventCreateWithFlags(&solved, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventRecord(solved, stream) == cudaSuccess && cudaStreamWaitEvent(cstream, solved, 0) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      if (rc == RS_OK) rc = RS_ERR_CUDA;
    }
    size_t col = 0;
    for (auto& r : cur) {
      double worst = 0;
      if (rc == RS_OK &&
          (r->ldx == n ? cudaMemcpyAsync(r->X, (const char*)dx[slot] + col * n * sb, n * sb * r->ncols,
                                         cudaMemcpyDeviceToHost, cstream)
                       : cudaMemcpy2DAsync(r->X, r->ldx * sb, (const char*)dx[slot] + col * n * sb, n * sb, n * sb,
                                           r->ncols, cudaMemcpyDeviceToHost, cstream)) != cudaSuccess) {
        cudaGetLastError();
        rc = RS_ERR_CUDA;
      }
      for (int c = 0; c < r->ncols; ++c, ++col) worst = std::max(worst, rel[col]);
      r->relres = worst;
      r->its = its;
    }
    cudaEventRecord(out_done[slot], cstream);
    Finished* f = new Finished{s, cur, rc, cur_cols};
    if (cudaLaunchHostFunc(cstream, finish_batch, f) != cudaSuccess) {   // complete here instead
      cudaGetLastError();
      cudaStreamSynchronize(cstream);
      finish_batch(f);
    }
    if (ok) cudaEventDestroy(solved);   // released once the recorded work completes
    cur.swap(next);
    cur_cols = next_cols;
    staged = next_staged;
    slot ^= 1;
  }
}

int add_worker(Server* s, rs_handle h, bool owned, int* id_out) {
  auto w = std::make_unique<Worker>();
  w->s = s;
  w->h = h;
  w->owned = owned;
  rs_stats_t st;
  RS_TRY(rs_stats(h, &st));
  w->n = st.n;
  w->cplx = static_cast<rs::Handle*>(reinterpret_cast<rs::Handle*>(h))->cplx;
  if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&w->cstream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return rs::fail(RS_ERR_CUDA, "rs_server: stream creation failed");
  }
  int dev = 0;
  cudaGetDevice(&dev);
  Worker* wp = w.get();
  w->th = std::thread([wp, dev] {
    cudaSetDevice(dev);
    wp->run();
  });
  w->id = (int)s->workers.size();
  *id_out = w->id;
  s->resident_bytes += handle_bytes(h);
  s->workers.push_back(std::move(w));
  return RS_OK;
}

void builder_loop(Server* s, int dev) {
  cudaSetDevice(dev);
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_build.wait(lk, [&] { return s->stop || !s->build_q.empty(); });
      if (s->stop && s->build_q.empty()) break;
      r = s->build_q.front();
      s->build_q.pop_front();
    }
    // admission: estimated footprint (same 2D proportion as resident ones) under the budget
    size_t est = (size_t)r->n * 1800 * 3;
    int rc = RS_OK;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      size_t free_b = 0, total_b = 0;
      cudaMemGetInfo(&free_b, &total_b);
      if (s->resident_bytes + est > s->budget || est > free_b) rc = RS_ERR_OOM;
    }
    rs_handle h = nullptr;
    if (rc == RS_OK) rc = rs_build(r->pts.data(), r->n, r->dim, &r->params, r->eps, r->leaf, st, &h);
    int id = -1;
    if (rc == RS_OK) {
      std::lock_guard<std::mutex> lk(s->mu);
      rc = add_worker(s, h, true, &id);
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r->result_hid = id;
      complete(s, r, rc);
    }
    s->cv_done.notify_all();
  }
  cudaStreamDestroy(st);
}

}  // namespace

struct rs_server_s : public Server {};

extern "C" {

int rs_server_create(int max_cols, int64_t hbm_budget_bytes, rs_server* out) {
  if (!out || max_cols < 1) return rs::fail(RS_ERR_ARG, "rs_server_create: bad arguments");
  rs_server_s* s = new rs_server_s();
  s->max_cols = max_cols;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return rs::fail(RS_ERR_CUDA, "rs_server_create: no device");
  }
  s->budget = hbm_budget_bytes > 0 ? (size_t)hbm_budget_bytes : (size_t)(free_b * 0.9);
  int dev = 0;
  cudaGetDevice(&dev);
  s->builder = std::thread(builder_loop, s, dev);
  *out = s;
  return RS_OK;
}

int rs_server_add_handle(rs_server s, rs_handle h, int* handle_id) {
  if (!s || !h || !handle_id) return rs::fail(RS_ERR_ARG, "rs_server_add_handle: null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  return add_worker(s, h, false, handle_id);
}

int rs_server_submit_solve(rs_server s, int handle_id, const void* B, int64_t ldb, int ncols, void* X, int64_t ldx,
                           double tol, int64_t* ticket) {
  if (!s || !B || !X || !ticket || ncols < 1) return rs::fail(RS_ERR_ARG, "rs_server_submit_solve: bad arguments");
  auto r = std::make_shared<Request>();
  r->kind = 0;
  r->hid = handle_id;
  r->B = B;
  r->ldb = ldb;
  r->X = X;
  r->ldx = ldx;
  r->ncols = ncols;
  r->tol = tol;
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (handle_id < 0 || handle_id >= (int)s->workers.size())
    return rs::fail(RS_ERR_ARG, "rs_server_submit_solve: unknown handle id %d", handle_id);
  Worker* w = s->workers[handle_id].get();
  if (ldb < w->n || ldx < w->n) return rs::fail(RS_ERR_ARG, "rs_server_submit_solve: leading dimension < N");
  if (ncols > s->max_cols) return rs::fail(RS_ERR_ARG, "rs_server_submit_solve: more columns than a batch holds");
  r->ticket = s->next_ticket++;
  s->reqs[r->ticket] = r;
  w->q.push_back(r);
  w->cv.notify_one();
  *ticket = r->ticket;
  return RS_OK;
}

int rs_server_submit_build(rs_server s, const double* pts, int64_t n, int dim, const rs_params* params, double eps,
                           int leaf, int64_t* ticket) {
  if (!s || !pts || !params || !ticket || n < 1) return rs::fail(RS_ERR_ARG, "rs_server_submit_build: bad arguments");
  auto r = std::make_shared<Request>();
  r->kind = 1;
  r->pts.assign(pts, pts + (size_t)n * dim);
  r->n = n;
  r->dim = dim;
  r->params = *params;
  if (params->kernel_id == RS_LAPLACE2D_DL) {   // copied like the points; the build reads the copies
    if (!params->normals || !params->curvature || dim != 2)
      return rs::fail(RS_ERR_ARG, "rs_server_submit_build: the double layer needs 2D points, normals and curvature");
    r->nrm.assign(params->normals, params->normals + (size_t)2 * n);
    r->kap.assign(params->curvature, params->curvature + (size_t)n);
    r->params.normals = r->nrm.data();
    r->params.curvature = r->kap.data();
  }
  r->eps = eps;
  r->leaf = leaf;
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  r->ticket = s->next_ticket++;
  s->reqs[r->ticket] = r;
  s->build_q.push_back(r);
  s->cv_build.notify_one();
  *ticket = r->ticket;
  return RS_OK;
}

int rs_server_wait(rs_server s, int64_t ticket, double timeout_s, int* status, double* latency_ms, double* relres,
                   int* result) {
  if (!s) return rs::fail(RS_ERR_ARG, "rs_server_wait: null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return rs::fail(RS_ERR_ARG, "rs_server_wait: unknown ticket");
  auto r = it->second;
  bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9),
                                [&] { return r->done; });
  if (!ok) return rs::fail(RS_ERR_TIMEOUT, "rs_server_wait: request %lld not done", (long long)ticket);
  if (status) *status = r->status;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  if (relres) *relres = r->relres;
  if (result) *result = r->kind == 1 ? r->result_hid : r->its;
  s->reqs.erase(it);
  return RS_OK;
}

int rs_server_stats(rs_server s, rs_server_stats_t* out) {
  if (!s || !out) return rs::fail(RS_ERR_ARG, "rs_server_stats: null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<double> v = s->lat_ms;
  std::sort(v.begin(), v.end());
  auto pct = [&](double p) {
    if (v.empty()) return 0.0;
    size_t i = (size_t)std::min<double>(v.size() - 1, std::ceil(p * v.size()) - 1);
    return v[i];
  };
  out->requests = (int64_t)v.size();
  out->rhs = s->rhs_done;
  out->batches = s->batches;
  out->mean_batch_cols = s->batches ? (double)s->batch_cols / s->batches : 0.0;
  out->p50_ms = pct(0.50);
  out->p99_ms = pct(0.99);
  out->elapsed_s = std::chrono::duration<double>(Clock::now() - s->t0).count();
  out->handles = (int)s->workers.size();
  out->resident_bytes = (int64_t)s->resident_bytes;
  return RS_OK;
}

int rs_server_reset_stats(rs_server s) {
  if (!s) return rs::fail(RS_ERR_ARG, "rs_server_reset_stats: null server");
  std::lock_guard<std::mutex> lk(s->mu);
  s->lat_ms.clear();
  s->rhs_done = s->batches = s->batch_cols = 0;
  s->t0 = Clock::now();
  return RS_OK;
}

int rs_server_destroy(rs_server s) {
  if (!s) return RS_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (auto& w : s->workers) w->cv.notify_all();
    s->cv_build.notify_all();
  }
  for (auto& w : s->workers)
    if (w->th.joinable()) w->th.join();
  if (s->builder.joinable()) s->builder.join();
  for (auto& w : s->workers) {
    if (w->cstream) cudaStreamSynchronize(w->cstream);   // last columns back and callbacks run
    if (w->stream) cudaStreamDestroy(w->stream);
    if (w->cstream) cudaStreamDestroy(w->cstream);
    for (int i = 0; i < 2; ++i) {
      if (w->db[i]) cudaFree(w->db[i]);
      if (w->dx[i]) cudaFree(w->dx[i]);
      if (w->in_done[i]) cudaEventDestroy(w->in_done[i]);
      if (w->out_done[i]) cudaEventDestroy(w->out_done[i]);
    }
    if (w->owned) rs_free(w->h);
  }
  delete s;
  return RS_OK;
}

int rs_server_handle(rs_server s, int handle_id, rs_handle* out) {
  if (!s || !out) return rs::fail(RS_ERR_ARG, "rs_server_handle: null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (handle_id < 0 || handle_id >= (int)s->workers.size()) return rs::fail(RS_ERR_ARG, "rs_server_handle: bad id");
  *out = s->workers[handle_id]->h;
  return RS_OK;
}

}  // extern "C"
