// Launch profiler: CUDA events around each kernel launch, grouped by
// category, with the launch's algorithmic bytes and flops counted on the
// host from the known block sizes.  Off unless rs_profile_enable(1).
#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "rs_internal.h"

namespace rs {

namespace {

struct Rec {
  int cat;
  cudaEvent_t e0, e1;
  double bytes, flops;
};

const char* kNames[P_NCAT] = {"tree", "id", "factor", "fp32_copy", "solve_up", "solve_down", "permute",
                              "fwd_proj", "fwd_dblock", "fwd_down", "residual", "misc", "solve_fp64",
                              "solve_fp32"};

std::mutex g_mu;
bool g_on = false;
bool g_tiles = false;   // also record the persistent launches' tile timelines
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
size_t g_next = 0;
std::vector<Rec> g_stack;

cudaEvent_t get_event() {
  if (g_next < g_pool.size()) return g_pool[g_next++];
  cudaEvent_t e;
  cudaEventCreate(&e);
  g_pool.push_back(e);
  ++g_next;
  return e;
}

}  // namespace

bool prof_on() { return g_on; }
bool prof_tiles_on() { return g_on && g_tiles; }

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void prof_begin(int cat, cudaStream_t st) {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Rec r{cat, get_event(), nullptr, 0.0, 0.0};
  cudaEventRecord(r.e0, st);
  g_stack.push_back(r);
}

void prof_end(int cat, cudaStream_t st, double bytes, double flops) {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_stack.empty()) return;
  Rec r = g_stack.back();
  g_stack.pop_back();
  r.cat = cat;
  r.e1 = get_event();
  r.bytes = bytes;
  r.flops = flops;
  cudaEventRecord(r.e1, st);
  g_recs.push_back(r);
}

void prof_amend(int cat, double bytes, double flops) {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto it = g_recs.rbegin(); it != g_recs.rend(); ++it)
    if (it->cat == cat) {
      it->bytes = bytes;
      it->flops = flops;
      return;
    }
}

// FMA throughput probe: every thread runs 8 independent FMA chains, so the
// pipe (not the FMA latency) bounds the rate.
template <class T>
__global__ void __launch_bounds__(256) k_fma_probe(T mul, T add, int iters, T* out) {
  T a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = a[i] * mul + add;
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
int fma_probe(double* gflops) {
  int dev = 0, nsm = 0;
  RS_CUDA(cudaGetDevice(&dev));
  RS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = nsm * 8, threads = 256, iters = sizeof(T) == 8 ? 1 << 12 : 1 << 15;
  T* out = nullptr;
  RS_CUDA(cudaMalloc((void**)&out, sizeof(T) * (size_t)blocks * threads));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int rc = RS_OK;
  for (int rep = 0; rep < 4 && rc == RS_OK; ++rep) {
    cudaEventRecord(e0);
    k_fma_probe<T><<<blocks, threads>>>((T)0.999999, (T)1e-7, iters, out);
    cudaEventRecord(e1);
    float ms = 0;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaGetLastError();
      rc = fail(RS_ERR_CUDA, "rs_probe_fma_peak: probe launch failed");
    } else if (rep > 0) {
      best = std::min(best, ms);   // the first launch pays one-time costs
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (rc == RS_OK) *gflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e9;
  return rc;
}

}  // namespace rs

extern "C" {

int rs_probe_fma_peak(int precision, double* gflops) {
  if (!gflops || (precision != RS_PREC_FP64 && precision != RS_PREC_FP32))
    return rs::fail(RS_ERR_ARG, "rs_probe_fma_peak: bad arguments");
  return precision == RS_PREC_FP64 ? rs::fma_probe<double>(gflops) : rs::fma_probe<float>(gflops);
}

int rs_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(rs::g_mu);
  rs::g_recs.clear();
  rs::g_stack.clear();
  rs::g_next = 0;
  rs::g_on = on != 0;
  rs::g_tiles = on == 2;
  return RS_OK;
}

int rs_profile_ncat(void) { return rs::P_NCAT; }

int64_t rs_launch_count(void) { return rs::g_launches.load(); }

int rs_profile_nrec(void) {
  std::lock_guard<std::mutex> lk(rs::g_mu);
  return (int)rs::g_recs.size();
}

int rs_profile_record(int i, int* cat, double* ms, double* bytes, double* flops) {
  std::lock_guard<std::mutex> lk(rs::g_mu);
  if (i < 0 || i >= (int)rs::g_recs.size()) return rs::fail(RS_ERR_ARG, "rs_profile_record: index out of range");
  const auto& r = rs::g_recs[i];
  float m = 0;
  if (cudaEventSynchronize(r.e1) != cudaSuccess || cudaEventElapsedTime(&m, r.e0, r.e1) != cudaSuccess) {
    cudaGetLastError();
    return rs::fail(RS_ERR_CUDA, "rs_profile_record: event timing failed");
  }
  if (cat) *cat = r.cat;
  if (ms) *ms = m;
  if (bytes) *bytes = r.bytes;
  if (flops) *flops = r.flops;
  return RS_OK;
}

int rs_profile_record_start(int i, double* start_ms) {
  std::lock_guard<std::mutex> lk(rs::g_mu);
  if (i < 0 || i >= (int)rs::g_recs.size()) return rs::fail(RS_ERR_ARG, "rs_profile_record_start: index out of range");
  float m = 0;
  const auto& r = rs::g_recs[i];
  if (cudaEventSynchronize(r.e1) != cudaSuccess || cudaEventElapsedTime(&m, rs::g_recs[0].e0, r.e0) != cudaSuccess) {
    cudaGetLastError();
    return rs::fail(RS_ERR_CUDA, "rs_profile_record_start: event timing failed");
  }
  if (start_ms) *start_ms = m;
  return RS_OK;
}

int rs_profile_read(int cat, double* ms, int64_t* launches, double* bytes, double* flops, const char** name) {
  if (cat < 0 || cat >= rs::P_NCAT) return rs::fail(RS_ERR_ARG, "rs_profile_read: bad category");
  std::lock_guard<std::mutex> lk(rs::g_mu);
  double t = 0, by = 0, fl = 0;
  int64_t n = 0;
  for (auto& r : rs::g_recs) {
    if (r.cat != cat) continue;
    float m = 0;
    if (cudaEventSynchronize(r.e1) != cudaSuccess || cudaEventElapsedTime(&m, r.e0, r.e1) != cudaSuccess) {
      cudaGetLastError();
      return rs::fail(RS_ERR_CUDA, "rs_profile_read: event timing failed");
    }
    t += m;
    by += r.bytes;
    fl += r.flops;
    ++n;
  }
  if (ms) *ms = t;
  if (launches) *launches = n;
  if (bytes) *bytes = by;
  if (flops) *flops = fl;
  if (name) *name = rs::kNames[cat];
  return RS_OK;
}

}  // extern "C"
