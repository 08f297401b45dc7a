// C ABI entry points and the host-side orchestration of build and solve.
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include <map>
#include <mutex>
#include <cstring>
#include "rs_internal.h"

// The opaque handle type of the C ABI is the runtime's Handle.
struct rs_handle_s : public rs::Handle {};

namespace rs {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

int fail(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

// Host-side fault injection (rs_set_fault): the n-th device allocation
// fails, or the next persistent solve waits on a target no tile reaches.
static std::atomic<long> g_fault_alloc{0};   // 0 = off, else allocations left before the failing one
static std::atomic<int> g_fault_wait{0};

bool take_wait_fault() { return g_fault_wait.exchange(0) != 0; }

static std::atomic<int> g_path_force{0};
static std::atomic<long long> g_path_count[PATH_N];
static std::atomic<int> g_solve_tile{-1};
int path_force() { return g_path_force.load(); }
int solve_tile_force() { return g_solve_tile.load(); }
void path_count(int which) {
  if (which >= 0 && which < PATH_N) g_path_count[which].fetch_add(1);
}

// Handle memory is carved out of chunks taken from the stream-ordered pool
// (whose memory the library keeps cached), so a build makes a handful of
// allocation calls instead of one per table, and a rebuild reuses the memory
// of a freed handle without going back to the driver.
int dalloc(Handle* h, void** p, size_t bytes) {
  constexpr size_t kChunk = 64u << 20, kAlign = 256;
  *p = nullptr;
  long left = g_fault_alloc.load();
  if (left > 0 && g_fault_alloc.fetch_sub(1) == 1)
    return fail(RS_ERR_OOM, "device allocation of %zu bytes: injected failure", bytes);
  bytes = (std::max<size_t>(bytes, 16) + kAlign - 1) & ~(kAlign - 1);
  auto take = [&](void** q, size_t sz) -> int {
    cudaError_t e = cudaMallocAsync(q, sz, h->bst);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *q = nullptr;
      return fail(e == cudaErrorMemoryAllocation ? RS_ERR_OOM : RS_ERR_CUDA, "device allocation of %zu bytes: %s", sz,
                  cudaGetErrorString(e));
    }
    h->allocs.push_back(*q);
    if (h->fst) {   // the factorization stream may use the block as well
      RS_CUDA(cudaEventRecord(h->aev, h->bst));
      RS_CUDA(cudaStreamWaitEvent(h->fst, h->aev, 0));
    }
    return RS_OK;
  };
  if (bytes > kChunk / 4) return take(p, bytes);   // large tables get their own block
  if (bytes > h->arena_left) {
    void* c = nullptr;
    RS_TRY(take(&c, kChunk));
    h->arena_cur = (char*)c;
    h->arena_left = kChunk;
  }
  *p = h->arena_cur;
  h->arena_cur += bytes;
  h->arena_left -= bytes;
  return RS_OK;
}

// Per-device table of log_tab (rs_common.cuh): (log c_i, 1 / c_i) for
// c_i = 1 + i/256, then log 2 as a 32-bit head and the rest, computed in long
// double on the host.  One 4 KiB allocation per device, kept for the process.
static std::mutex g_logtab_mu;
static std::map<int, double*> g_logtab;

static int log_table(const double** out) {
  int dev = 0;
  RS_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_logtab_mu);
  auto it = g_logtab.find(dev);
  if (it != g_logtab.end()) {
    *out = it->second;
    return RS_OK;
  }
  std::vector<double> t(2 * (rs::LOGTAB_N + 1));
  for (int i = 0; i < rs::LOGTAB_N; ++i) {
    const long double c = 1.0L + (long double)i / rs::LOGTAB_N;
    t[2 * i] = (double)logl(c);
    t[2 * i + 1] = (double)(1.0L / c);
  }
  const long double ln2 = logl(2.0L);
  uint64_t bits;
  double head = (double)ln2;
  std::memcpy(&bits, &head, sizeof(bits));
  bits &= ~((uint64_t(1) << 21) - 1);   // 32 significant bits: e * head is exact for |e| < 2^21
  std::memcpy(&head, &bits, sizeof(bits));
  t[2 * rs::LOGTAB_N] = head;
  t[2 * rs::LOGTAB_N + 1] = (double)(ln2 - (long double)head);
  double* d = nullptr;
  RS_CUDA(cudaMalloc((void**)&d, sizeof(double) * t.size()));
  RS_CUDA(cudaMemcpy(d, t.data(), sizeof(double) * t.size(), cudaMemcpyHostToDevice));
  g_logtab[dev] = d;
  *out = d;
  return RS_OK;
}

__global__ void k_green(rs::KParams kp, const double* s2, int64_t n, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (kp.kind == RS_HELMHOLTZ2D || kp.kind == RS_HELMHOLTZ3D) {
    const rs::c128 g = rs::green_cplx(kp.kind, kp.kwave, sqrt(s2[i]));
    out[2 * i] = g.re;
    out[2 * i + 1] = g.im;
  } else {
    out[i] = rs::green_real_s2(kp, s2[i]);
  }
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static void destroy(rs_handle_s* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  free_pers(h);
  for (void* p : h->allocs) cudaFreeAsync(p, 0);
  for (auto& w : h->work) {
    for (void* p : w.v) if (p) cudaFree(p);
    for (void* p : w.u) if (p) cudaFree(p);
    if (w.vin) cudaFree(w.vin);
  }
  for (void* p : h->fz) if (p) cudaFree(p);
  for (void* p : h->fy) if (p) cudaFree(p);
  for (void* p : {h->r64, h->x64, h->b64}) if (p) cudaFree(p);
  if (h->colnorm) cudaFree(h->colnorm);
  delete h;
}

// Staging of caller buffers: device pointers are used as they are, host
// buffers go through a device copy (N x nrhs, ld = N).
struct Staged {
  void* d = nullptr;
  int64_t ld = 0;
  bool owned = false;
};

static int stage_in(const void* p, int64_t ld, int64_t N, int nrhs, size_t sb, cudaStream_t st, Staged* s) {
  if (is_device_ptr(p)) {
    s->d = const_cast<void*>(p);
    s->ld = ld;
    return RS_OK;
  }
  RS_CUDA(cudaMallocAsync(&s->d, sb * (size_t)N * nrhs, st));
  s->owned = true;
  s->ld = N;
  if (ld == N)   // contiguous: one plain copy (the pitched form ran at half the link's rate)
    RS_CUDA(cudaMemcpyAsync(s->d, p, sb * (size_t)N * nrhs, cudaMemcpyHostToDevice, st));
  else
    RS_CUDA(cudaMemcpy2DAsync(s->d, sb * N, p, sb * ld, sb * N, nrhs, cudaMemcpyHostToDevice, st));
  return RS_OK;
}

static int stage_out_alloc(void* p, int64_t ld, int64_t N, int nrhs, size_t sb, cudaStream_t st, Staged* s) {
  if (is_device_ptr(p)) {
    s->d = p;
    s->ld = ld;
    return RS_OK;
  }
  RS_CUDA(cudaMallocAsync(&s->d, sb * (size_t)N * nrhs, st));
  s->owned = true;
  s->ld = N;
  return RS_OK;
}

static int stage_out_finish(void* p, int64_t ld, int64_t N, int nrhs, size_t sb, cudaStream_t st, Staged* s) {
  if (s->owned) {
    if (ld == N)
      RS_CUDA(cudaMemcpyAsync(p, s->d, sb * (size_t)N * nrhs, cudaMemcpyDeviceToHost, st));
    else
      RS_CUDA(cudaMemcpy2DAsync(p, sb * ld, s->d, sb * N, sb * N, nrhs, cudaMemcpyDeviceToHost, st));
  }
  return RS_OK;
}

static void release(Staged* s, cudaStream_t st) {
  if (s->owned && s->d) cudaFreeAsync(s->d, st);
  s->d = nullptr;
}

// The double layer's normals (2 x N, point-major) and curvatures (N) in
// tree order: dlg = [normal x | normal y | curvature], N each.
__global__ void k_permute_dlayer(const double* nrm, const double* kap, const int* perm, int64_t n, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t src = perm[i];
  out[i] = nrm[2 * src];
  out[n + i] = nrm[2 * src + 1];
  out[2 * n + i] = kap[src];
}

static int load_dlayer(Handle* h, const double* nrm, const double* kap, cudaStream_t st) {
  const int64_t n = h->N;
  const double* dn = nrm;
  const double* dk = kap;
  double *tn = nullptr, *tk = nullptr;
  if (!is_device_ptr(nrm)) {
    RS_TRY(dalloc_t(h, &tn, (size_t)2 * n));
    RS_CUDA(cudaMemcpyAsync(tn, nrm, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, st));
    dn = tn;
  }
  if (!is_device_ptr(kap)) {
    RS_TRY(dalloc_t(h, &tk, (size_t)n));
    RS_CUDA(cudaMemcpyAsync(tk, kap, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    dk = tk;
  }
  RS_TRY(dalloc_t(h, &h->dlg, (size_t)3 * n));
  k_permute_dlayer<<<div_up(n, 256), 256, 0, st>>>(dn, dk, h->perm, n, h->dlg);
  RS_CHECK_LAUNCH();
  return RS_OK;
}

static int check_handle(rs_handle h) {
  if (!h) return fail(RS_ERR_ARG, "null handle");
  return RS_OK;
}

}  // namespace rs

using namespace rs;

extern "C" {

const char* rs_last_error(void) { return rs::g_err.c_str(); }

int rs_green(int kernel_id, double k_wave, const double* s2, int64_t n, double* out) {
  rs::g_err.clear();
  if (kernel_id < RS_LAPLACE2D || kernel_id > RS_HELMHOLTZ3D || n < 0 || (n > 0 && (!s2 || !out)))
    return fail(RS_ERR_ARG, "rs_green: bad arguments");
  if (n == 0) return RS_OK;
  rs::KParams kp{};
  kp.kind = kernel_id;
  kp.w = 1.0;
  kp.kwave = k_wave;
  RS_TRY(log_table(&kp.logtab));
  const int64_t nout = (kernel_id == RS_HELMHOLTZ2D || kernel_id == RS_HELMHOLTZ3D) ? 2 * n : n;
  double *ds = nullptr, *dout = nullptr;
  int rc = RS_OK;
  if (cudaMalloc((void**)&ds, sizeof(double) * n) || cudaMalloc((void**)&dout, sizeof(double) * nout)) {
    rc = fail(RS_ERR_OOM, "rs_green: allocation failed");
  } else if (cudaMemcpy(ds, s2, sizeof(double) * n, cudaMemcpyHostToDevice)) {
    rc = fail(RS_ERR_CUDA, "rs_green: copy failed");
  } else {
    k_green<<<(unsigned)((n + 255) / 256), 256>>>(kp, ds, n, dout);
    rs::count_launch();
    if (cudaGetLastError() || cudaMemcpy(out, dout, sizeof(double) * nout, cudaMemcpyDeviceToHost))
      rc = fail(RS_ERR_CUDA, "rs_green: evaluation failed");
  }
  cudaGetLastError();
  if (ds) cudaFree(ds);
  if (dout) cudaFree(dout);
  return rc;
}

const char* rs_version(void) { return "rs-gb300 0.1 (sm_103a)"; }

int rs_build(const double* pts, int64_t n, int dim, const rs_params* params, double eps, int leaf, void* stream,
             rs_handle* out) {
  rs::g_err.clear();
  if (!out) return fail(RS_ERR_ARG, "rs_build: out is null");
  *out = nullptr;
  if (!pts || !params) return fail(RS_ERR_ARG, "rs_build: null pointer argument");
  if (n < 1 || n > (int64_t)1 << 30) return fail(RS_ERR_ARG, "rs_build: N=%lld out of range", (long long)n);
  if (dim != 2 && dim != 3) return fail(RS_ERR_ARG, "rs_build: dim must be 2 or 3");
  if (params->kernel_id < RS_LAPLACE2D || params->kernel_id > RS_LAPLACE2D_DL)
    return fail(RS_ERR_ARG, "rs_build: unknown kernel_id %d", params->kernel_id);
  const bool helm = params->kernel_id == RS_HELMHOLTZ2D || params->kernel_id == RS_HELMHOLTZ3D;
  const bool dl = params->kernel_id == RS_LAPLACE2D_DL;
  if ((params->kernel_id == RS_LAPLACE3D || params->kernel_id == RS_HELMHOLTZ3D) != (dim == 3))
    return fail(RS_ERR_ARG, "rs_build: kernel %d does not match dim %d", params->kernel_id, dim);
  if (!(eps > 0.0 && eps < 1.0)) return fail(RS_ERR_ARG, "rs_build: eps must be in (0, 1)");
  if (leaf < 1) return fail(RS_ERR_ARG, "rs_build: leaf must be >= 1");
  if (dl) {
    if (!(params->weight != 0.0) || !std::isfinite(params->weight))
      return fail(RS_ERR_ARG, "rs_build: the double layer needs a finite nonzero weight");
    if (!params->normals || !params->curvature)
      return fail(RS_ERR_ARG, "rs_build: the double layer needs normals and curvature");
    if (params->id_oversample > 0 || params->id_arith != RS_ID_FP64)
      return fail(RS_ERR_ARG, "rs_build: the double layer runs the deterministic FP64 ID");
  } else if (!(params->weight > 0.0) || !std::isfinite(params->weight)) {
    return fail(RS_ERR_ARG, "rs_build: weight must be > 0");
  }
  if (params->proxy_n < 1) return fail(RS_ERR_ARG, "rs_build: proxy_n must be >= 1");
  if (!(params->proxy_ratio > 1.0)) return fail(RS_ERR_ARG, "rs_build: proxy_ratio must be > 1");
  if (params->id_arith != RS_ID_FP64 && params->id_arith != RS_ID_DFLOAT)
    return fail(RS_ERR_ARG, "rs_build: unknown id_arith %d", params->id_arith);
  if (params->id_oversample < 0 || params->id_oversample > 512)
    return fail(RS_ERR_ARG, "rs_build: id_oversample must be in 0..512");
  if (params->id_oversample > 0 && params->id_arith == RS_ID_DFLOAT)
    return fail(RS_ERR_ARG, "rs_build: the randomized ID runs the FP64 pivoted QR (id_arith must be RS_ID_FP64)");
  if (dim == 3) {
    int g = (int)std::lround(std::sqrt(params->proxy_n / 6.0));
    if (6 * g * g != params->proxy_n) return fail(RS_ERR_ARG, "rs_build: 3D proxy_n must be 6 g^2");
  }
  if (helm && !(params->k_wave > 0.0))
    return fail(RS_ERR_ARG, "rs_build: Helmholtz needs k_wave > 0");

  cudaStream_t st = (cudaStream_t)stream;
  {
    // keep stream-ordered allocations cached between calls (the default
    // release threshold returns them to the driver at every synchronize)
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
  }
  rs_handle_s* h = new rs_handle_s();
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(RS_ERR_CUDA, "rs_build: no current CUDA device");
  }
  h->dim = dim;
  h->N = n;
  h->kp.kind = params->kernel_id;
  h->kp.w = params->weight;
  h->kp.kwave = params->k_wave;
  {
    const int rc0 = log_table(&h->kp.logtab);
    if (rc0 != RS_OK) {
      delete h;
      return rc0;
    }
  }
  h->cplx = helm;
  h->nonsym = dl;
  h->nproxy = params->proxy_n;
  h->ratio = params->proxy_ratio;
  h->id_df = params->id_arith == RS_ID_DFLOAT;
  h->id_p = params->id_oversample;
  h->id_seed = params->id_seed;
  h->eps = eps;
  h->leaf = leaf;

  cudaEvent_t e0, e1, ej;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventCreateWithFlags(&ej, cudaEventDisableTiming);
  cudaEventRecord(e0, st);
  h->bst = st;
  int rc = RS_OK;
  // the skeletonization (the critical path) runs on a high-priority stream
  // `is`, the factorization behind it on a low-priority stream fs
  cudaStream_t fs = nullptr, is = nullptr;
  do {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&fs, cudaStreamNonBlocking, least) != cudaSuccess ||
        cudaStreamCreateWithPriority(&is, cudaStreamNonBlocking, greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->aev, cudaEventDisableTiming) != cudaSuccess) {
      rc = fail(RS_ERR_CUDA, "rs_build: stream creation failed");
      break;
    }
    h->fst = fs;
    if ((rc = dalloc_t(h, &h->status, 4)) != RS_OK) break;
    if (cudaMemsetAsync(h->status, 0, sizeof(int) * 4, st) != cudaSuccess) { rc = fail(RS_ERR_CUDA, "memset"); break; }
    const double* dp = pts;
    double* tmp = nullptr;
    if (!is_device_ptr(pts)) {
      if ((rc = dalloc_t(h, &tmp, (size_t)n * dim)) != RS_OK) break;
      if (cudaMemcpyAsync(tmp, pts, sizeof(double) * n * dim, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        rc = fail(RS_ERR_CUDA, "copy of points failed");
        break;
      }
      dp = tmp;
    }
    if ((rc = build_tree(h, dp, st)) != RS_OK) break;
    if (dl && (rc = load_dlayer(h, params->normals, params->curvature, st)) != RS_OK) break;
    // is and fs start after everything queued on st so far (tree, status
    // words); allocations are ordered on is from here on
    if (cudaEventRecord(ej, st) != cudaSuccess || cudaStreamWaitEvent(fs, ej, 0) != cudaSuccess ||
        cudaStreamWaitEvent(is, ej, 0) != cudaSuccess) {
      rc = fail(RS_ERR_CUDA, "rs_build: stream ordering failed");
      break;
    }
    h->bst = is;
    for (int d = h->L; d >= 1 && rc == RS_OK; --d) rc = skeletonize_level(h, d, is, fs);
    if (rc != RS_OK) break;
    if ((rc = factor_root(h, is, fs)) != RS_OK) break;
    if (cudaEventRecord(ej, fs) != cudaSuccess || cudaStreamWaitEvent(st, ej, 0) != cudaSuccess ||
        cudaEventRecord(ej, is) != cudaSuccess || cudaStreamWaitEvent(st, ej, 0) != cudaSuccess) {
      rc = fail(RS_ERR_CUDA, "rs_build: stream ordering failed");
      break;
    }
    h->fst = nullptr;
    h->bst = st;
    if ((rc = check_factor_status(h, st)) != RS_OK) break;
    if ((rc = make_fp32_copies(h, st)) != RS_OK) break;
    if ((rc = make_fwd_blocks(h, st)) != RS_OK) break;
  } while (0);
  h->fst = nullptr;
  h->bst = st;
  for (cudaStream_t x : {fs, is})
    if (x) {
      cudaStreamSynchronize(x);
      cudaStreamDestroy(x);
    }
  if (h->aev) {
    cudaEventDestroy(h->aev);
    h->aev = nullptr;
  }
  cudaEventRecord(e1, st);
  cudaError_t se = cudaStreamSynchronize(st);
  if (rc == RS_OK && se != cudaSuccess) rc = fail(RS_ERR_CUDA, "rs_build: %s", cudaGetErrorString(se));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(ej);
  if (rc != RS_OK) {
    std::string keep = rs::g_err;
    destroy(h);
    rs::g_err = keep;
    return rc;
  }
  h->build_ms = ms;
  *out = h;
  return RS_OK;
}

int rs_solve(rs_handle h, int precision, const void* B, int64_t ldb, int nrhs, void* X, int64_t ldx, void* stream) {
  rs::g_err.clear();
  RS_TRY(check_handle(h));
  if (!B || !X) return fail(RS_ERR_ARG, "rs_solve: null buffer");
  if (nrhs < 1 || ldb < h->N || ldx < h->N) return fail(RS_ERR_ARG, "rs_solve: bad nrhs or leading dimension");
  if (precision != RS_PREC_FP64 && precision != RS_PREC_FP32) return fail(RS_ERR_ARG, "rs_solve: bad precision");
  cudaStream_t st = (cudaStream_t)stream;
  size_t sb = h->cplx ? sizeof(c128) : sizeof(double);
  Staged sB, sX;
  int rc = stage_in(B, ldb, h->N, nrhs, sb, st, &sB);
  if (rc == RS_OK) rc = stage_out_alloc(X, ldx, h->N, nrhs, sb, st, &sX);
  if (rc == RS_OK) rc = solve_pers_device(h, precision, sB.d, sB.ld, nrhs, sX.d, sX.ld, st);
  if (rc == RS_OK) rc = stage_out_finish(X, ldx, h->N, nrhs, sb, st, &sX);
  cudaError_t e = cudaStreamSynchronize(st);
  release(&sB, st);
  release(&sX, st);
  if (rc == RS_OK && e != cudaSuccess) rc = fail(RS_ERR_CUDA, "rs_solve: %s", cudaGetErrorString(e));
  if (rc == RS_OK) rc = pers_check(h);
  return rc;
}

int rs_solve_noalloc(rs_handle h, int precision, const void* B, int64_t ldb, int nrhs, void* X, int64_t ldx,
                     void* stream) {
  rs::g_err.clear();
  RS_TRY(check_handle(h));
  if (!B || !X) return fail(RS_ERR_ARG, "rs_solve_noalloc: null buffer");
  if (nrhs < 1 || ldb < h->N || ldx < h->N) return fail(RS_ERR_ARG, "rs_solve_noalloc: bad nrhs or leading dimension");
  if (precision != RS_PREC_FP64 && precision != RS_PREC_FP32)
    return fail(RS_ERR_ARG, "rs_solve_noalloc: bad precision");
  if (!is_device_ptr(B) || !is_device_ptr(X))
    return fail(RS_ERR_ARG, "rs_solve_noalloc: B and X must be device memory (host buffers would need staging)");
  {
    // the scratch array's address is looked up for the current device, the
    // factors live on the handle's: the two must be the same GPU
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
      cudaGetLastError();
      return fail(RS_ERR_CUDA, "rs_solve_noalloc: no current CUDA device");
    }
    if (dev != h->device)
      return fail(RS_ERR_ARG, "rs_solve_noalloc: current device %d is not the handle's device %d", dev, h->device);
  }
  cudaStream_t st = (cudaStream_t)stream;
  int rc = solve_noalloc_device(h, precision, B, ldb, nrhs, X, ldx, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (rc == RS_OK && e != cudaSuccess) rc = fail(RS_ERR_CUDA, "rs_solve_noalloc: %s", cudaGetErrorString(e));
  return rc;
}

int rs_matvec(rs_handle h, const void* X, int64_t ldx, int nrhs, void* Y, int64_t ldy, void* stream) {
  rs::g_err.clear();
  RS_TRY(check_handle(h));
  if (!X || !Y) return fail(RS_ERR_ARG, "rs_matvec: null buffer");
  if (nrhs < 1 || ldx < h->N || ldy < h->N) return fail(RS_ERR_ARG, "rs_matvec: bad nrhs or leading dimension");
  cudaStream_t st = (cudaStream_t)stream;
  size_t sb = h->cplx ? sizeof(c128) : sizeof(double);
  Staged sX, sY;
  int rc = stage_in(X, ldx, h->N, nrhs, sb, st, &sX);
  if (rc == RS_OK) rc = stage_out_alloc(Y, ldy, h->N, nrhs, sb, st, &sY);
  if (rc == RS_OK) rc = matvec_device(h, sX.d, sX.ld, nrhs, sY.d, sY.ld, st);
  if (rc == RS_OK) rc = stage_out_finish(Y, ldy, h->N, nrhs, sb, st, &sY);
  cudaError_t e = cudaStreamSynchronize(st);
  release(&sX, st);
  release(&sY, st);
  if (rc == RS_OK && e != cudaSuccess) rc = fail(RS_ERR_CUDA, "rs_matvec: %s", cudaGetErrorString(e));
  return rc;
}

int rs_solve_refined(rs_handle h, const void* B, int64_t ldb, int nrhs, void* X, int64_t ldx, double tol,
                     int max_it, int* its_out, double* relres_out, void* stream) {
  rs::g_err.clear();
  RS_TRY(check_handle(h));
  if (!B || !X) return fail(RS_ERR_ARG, "rs_solve_refined: null buffer");
  if (nrhs < 1 || ldb < h->N || ldx < h->N) return fail(RS_ERR_ARG, "rs_solve_refined: bad nrhs or ld");
  if (!(tol > 0.0) || max_it < 0) return fail(RS_ERR_ARG, "rs_solve_refined: bad tol or max_it");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t N = h->N;
  size_t sb = h->cplx ? sizeof(c128) : sizeof(double);
  Staged sB, sX;
  int rc = stage_in(B, ldb, N, nrhs, sb, st, &sB);
  if (rc != RS_OK) return rc;
  // contiguous copies b (ld N), x, r, d
  void *b = nullptr, *x = nullptr, *r = nullptr, *d = nullptr;
  double* nrm = nullptr;
  size_t bytes = sb * (size_t)N * nrhs;
  std::vector<double> hb(nrhs), hr(nrhs);
  int its = 0;
  do {
    if (cudaMallocAsync(&b, bytes, st) || cudaMallocAsync(&x, bytes, st) || cudaMallocAsync(&r, bytes, st) ||
        cudaMallocAsync(&d, bytes, st) || cudaMallocAsync((void**)&nrm, sizeof(double) * 2 * nrhs, st)) {
      rc = fail(RS_ERR_OOM, "rs_solve_refined: workspace allocation failed");
      break;
    }
    if (cudaMemcpy2DAsync(b, sb * N, sB.d, sb * sB.ld, sb * N, nrhs, cudaMemcpyDeviceToDevice, st)) {
      rc = fail(RS_ERR_CUDA, "copy");
      break;
    }
    if ((rc = colnorm2_device(h, b, nrhs, nrm + nrhs, st)) != RS_OK) break;
    if ((rc = solve_pers_device(h, RS_PREC_FP32, b, N, nrhs, x, N, st)) != RS_OK) break;
    cudaMemcpyAsync(hb.data(), nrm + nrhs, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st);
    // r_0 = b - A x_0 with double-float products (complex kernels: complex
    // double-float); later residuals by the update r_{j+1} = r_j - A d_j (float /
    // complex float products on the small correction), all from the stored
    // forward factors.
    bool first = true;
    for (;;) {
      if (first && (rc = residual_df(h, (const double*)b, (const double*)x, (double*)r, nrhs, true, st)) != RS_OK)
        break;
      first = false;
      if ((rc = colnorm2_device(h, r, nrhs, nrm, st)) != RS_OK) break;
      cudaMemcpyAsync(hr.data(), nrm, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
      if ((rc = pers_check(h)) != RS_OK) break;
      bool done = true;
      for (int c = 0; c < nrhs; ++c) {
        double rel = hb[c] > 0 ? std::sqrt(hr[c] / hb[c]) : std::sqrt(hr[c]);
        if (!std::isfinite(rel)) { rc = fail(RS_ERR_NAN, "rs_solve_refined: non-finite residual"); break; }
        if (relres_out) relres_out[c] = rel;
        if (rel > tol) done = false;
      }
      if (rc != RS_OK || done || its >= max_it) break;
      if ((rc = solve_pers_device(h, RS_PREC_FP32, r, N, nrhs, d, N, st)) != RS_OK) break;
      if ((rc = axpy_lowp_device(h, x, d, nrhs, st)) != RS_OK) break;
      if ((rc = residual_df(h, (const double*)r, (const double*)d, (double*)r, nrhs, false, st)) != RS_OK) break;
      ++its;
    }
    if (rc != RS_OK) break;
    if ((rc = stage_out_alloc(X, ldx, N, nrhs, sb, st, &sX)) != RS_OK) break;
    if (cudaMemcpy2DAsync(sX.d, sb * sX.ld, x, sb * N, sb * N, nrhs, cudaMemcpyDeviceToDevice, st)) {
      rc = fail(RS_ERR_CUDA, "copy");
      break;
    }
    rc = stage_out_finish(X, ldx, N, nrhs, sb, st, &sX);
  } while (0);
  cudaError_t e = cudaStreamSynchronize(st);
  for (void* p : {b, x, r, d, (void*)nrm}) if (p) cudaFreeAsync(p, st);
  release(&sB, st);
  release(&sX, st);
  cudaStreamSynchronize(st);
  if (rc == RS_OK && e != cudaSuccess) rc = fail(RS_ERR_CUDA, "rs_solve_refined: %s", cudaGetErrorString(e));
  if (its_out) *its_out = its;
  return rc;
}

int rs_profile_tiles(rs_handle h, int mode, int nrhs, int64_t cap, int* kind, int* depth, int* row0, int* ncol,
                     double* t_claim_us, double* t_start_us, double* t_end_us, int64_t* count) {
  RS_TRY(check_handle(h));
  if (mode < 0 || mode > 3 || nrhs < 1 || cap < 0) return fail(RS_ERR_ARG, "rs_profile_tiles: bad arguments");
  return rs::tile_trace(h, mode, nrhs, cap, kind, depth, row0, ncol, t_claim_us, t_start_us, t_end_us, count);
}

int rs_stats(rs_handle h, rs_stats_t* out) {
  RS_TRY(check_handle(h));
  if (!out) return fail(RS_ERR_ARG, "rs_stats: null output");
  out->n = h->N;
  out->dim = h->dim;
  out->depth = h->L;
  out->top_skeletons = h->lv[0].ntot;
  out->factor_scalars = h->factor_scalars;
  out->factor_bytes = h->factor_scalars * (int64_t)(h->cplx ? sizeof(c128) : sizeof(double));
  out->build_ms = h->build_ms;
  int mn = 0, mm = 0, mk = 0;
  for (auto& lv : h->lv) {
    mn = std::max(mn, lv.maxn);
    mm = std::max(mm, lv.maxm);
    mk = std::max(mk, lv.maxk);
  }
  out->max_box_n = mn;
  out->max_box_m = mm;
  out->max_rank = mk;
  return RS_OK;
}

int rs_tree_perm(rs_handle h, int64_t* perm) {
  RS_TRY(check_handle(h));
  if (!perm) return fail(RS_ERR_ARG, "rs_tree_perm: null output");
  std::vector<int> p(h->N);
  RS_CUDA(cudaMemcpy(p.data(), h->perm, sizeof(int) * h->N, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < h->N; ++i) perm[i] = p[i];
  return RS_OK;
}

int rs_tree_level(rs_handle h, int level, int* nbox_out, int64_t* begin, int* parent, int* ncoll, int* coll) {
  RS_TRY(check_handle(h));
  if (level < 0 || level > h->L) return fail(RS_ERR_ARG, "rs_tree_level: level %d out of range", level);
  const Level& lv = h->lv[level];
  if (nbox_out) *nbox_out = lv.nbox;
  for (int b = 0; b < lv.nbox; ++b) {
    if (begin) begin[b] = lv.h_begin[b];
    if (parent) parent[b] = lv.h_parent[b];
    if (ncoll) ncoll[b] = lv.h_ncoll[b];
  }
  if (coll) std::copy(lv.h_coll.begin(), lv.h_coll.end(), coll);
  return RS_OK;
}

int rs_box_ranks(rs_handle h, int level, int* n, int* k) {
  RS_TRY(check_handle(h));
  if (level < 1 || level > h->L) return fail(RS_ERR_ARG, "rs_box_ranks: level %d out of range", level);
  const Level& lv = h->lv[level];
  for (int b = 0; b < lv.nbox; ++b) {
    if (n) n[b] = lv.h_n[b];
    if (k) k[b] = lv.h_k[b];
  }
  return RS_OK;
}

int rs_set_fault(const char* spec) {
  rs::g_err.clear();
  if (!spec || !*spec || std::string(spec) == "off") {
    g_fault_alloc = 0;
    g_fault_wait = 0;
    return RS_OK;
  }
  std::string s(spec);
  if (s == "wait") {
    g_fault_wait = 1;
    return RS_OK;
  }
  if (s.rfind("alloc:", 0) == 0) {
    long n = std::atol(s.c_str() + 6);
    if (n < 1) return fail(RS_ERR_ARG, "rs_set_fault: alloc:n needs n >= 1");
    g_fault_alloc = n;
    return RS_OK;
  }
  return fail(RS_ERR_ARG, "rs_set_fault: unknown fault '%s'", spec);
}

// Points (dim x n, point-major, host or device) to per-axis device arrays.
__global__ void k_pts_soa(const double* in, int dim, int64_t n, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int d = 0; d < dim; ++d) out[d * n + i] = in[i * dim + d];
}

int rs_gmres_patches(int npatch, const rs_handle* patches, const double* pts, const void* B, void* X, double tol,
                     int max_it, int restart, int precondition, int* its_out, double* relres_out, void* stream) {
  rs::g_err.clear();
  if (npatch < 1 || !patches || !pts || !B || !X) return fail(RS_ERR_ARG, "rs_gmres_patches: null or empty argument");
  if (!(tol > 0.0) || max_it < 1 || restart < 1 || restart > 200)
    return fail(RS_ERR_ARG, "rs_gmres_patches: need tol > 0, max_it >= 1, 1 <= restart <= 200");
  std::vector<Handle*> hs(npatch);
  int64_t n = 0;
  for (int i = 0; i < npatch; ++i) {
    RS_TRY(check_handle(patches[i]));
    hs[i] = patches[i];
    const Handle* a = hs[0];
    const Handle* b = hs[i];
    if (b->kp.kind != a->kp.kind || b->kp.kwave != a->kp.kwave || b->dim != a->dim || b->cplx != a->cplx)
      return fail(RS_ERR_ARG, "rs_gmres_patches: patches must share the kernel, wavenumber and dimension");
    if (b->nonsym) return fail(RS_ERR_ARG, "rs_gmres_patches: the coupled apply takes the Green's functions only");
    n += b->N;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int dim = hs[0]->dim;
  const size_t sb = hs[0]->cplx ? sizeof(c128) : sizeof(double);
  Staged sP, sB, sX;
  double* soa = nullptr;
  int rc = stage_in(pts, dim, dim, (int)n, sizeof(double), st, &sP);   // dim x n, one "column" per point
  if (rc == RS_OK) rc = stage_in(B, n, n, 1, sb, st, &sB);
  if (rc == RS_OK) rc = stage_out_alloc(X, n, n, 1, sb, st, &sX);
  if (rc == RS_OK && cudaMallocAsync((void**)&soa, sizeof(double) * 3 * n, st) != cudaSuccess) {
    cudaGetLastError();
    rc = fail(RS_ERR_OOM, "rs_gmres_patches: point buffer allocation failed");
  }
  if (rc == RS_OK) {
    k_pts_soa<<<(int)std::min<int64_t>(4096, (n + 255) / 256), 256, 0, st>>>((const double*)sP.d, dim, n, soa);
    RS_CHECK_LAUNCH();
    rc = gmres_patches_device(npatch, hs.data(), soa, sB.d, sX.d, tol, max_it, restart, precondition, its_out,
                              relres_out, st);
  }
  if (rc == RS_OK) rc = stage_out_finish(X, n, n, 1, sb, st, &sX);
  cudaError_t e = cudaStreamSynchronize(st);
  if (soa) cudaFreeAsync(soa, st);
  release(&sP, st);
  release(&sB, st);
  release(&sX, st);
  cudaStreamSynchronize(st);
  if (rc == RS_OK && e != cudaSuccess) rc = fail(RS_ERR_CUDA, "rs_gmres_patches: %s", cudaGetErrorString(e));
  return rc;
}

int rs_set_path(const char* spec) {
  rs::g_err.clear();
  if (!spec || !*spec) {
    g_path_force = 0;
    g_solve_tile = -1;
    return RS_OK;
  }
  static const std::pair<const char*, int> names[] = {
      {"off", 0},
      {"id:big", PF_ID_BIG},
      {"id:coop", PF_ID_BIG | PF_ID_NOCLUSTER},
      {"id:step", PF_ID_BIG | PF_ID_NOCLUSTER | PF_ID_NOCOOP},
      {"factor:big", PF_FACTOR_BIG},
      {"gj:blocked", PF_GJ_NOCLUSTER},
      {"gj:coop", PF_GJ_NOCLUSTER | PF_GJ_NOBLOCKED},
      {"gj:step", PF_GJ_NOCLUSTER | PF_GJ_NOBLOCKED | PF_GJ_NOCOOP}};
  int f = 0, tile = -1;
  std::string s(spec);
  size_t pos = 0;
  while (pos <= s.size()) {
    size_t e = s.find(',', pos);
    if (e == std::string::npos) e = s.size();
    const std::string tok = s.substr(pos, e - pos);
    bool found = false;
    if (tok.rfind("tile:", 0) == 0) {
      int tm = 0, tn = 0;
      const std::string v = tok.substr(5);
      if (v == "warp") tile = 0;
      else if (sscanf(v.c_str(), "%dx%d", &tm, &tn) == 2 &&
               (((tm == 32 || tm == 64) && (tn == 32 || tn == 64)) ||
                (tm == 128 && (tn == 64 || tn == 128 || tn == 256))))
        tile = tm * 1000 + tn;
      else
        return fail(RS_ERR_ARG, "rs_set_path: unknown tile '%s'", v.c_str());
      pos = e + 1;
      continue;
    }
    for (auto& nm : names)
      if (tok == nm.first) {
        f |= nm.second;
        found = true;
      }
    if (!found) return fail(RS_ERR_ARG, "rs_set_path: unknown path '%s'", tok.c_str());
    pos = e + 1;
  }
  g_path_force = f;
  g_solve_tile = tile;
  return RS_OK;
}

int rs_path_counts(int64_t* counts, int cap, int reset) {
  rs::g_err.clear();
  if (cap < 0 || (cap > 0 && !counts)) return fail(RS_ERR_ARG, "rs_path_counts: bad output");
  for (int i = 0; i < PATH_N; ++i) {
    const long long v = reset ? g_path_count[i].exchange(0) : g_path_count[i].load();
    if (i < cap) counts[i] = v;
  }
  return PATH_N;
}

int rs_free(rs_handle h) {
  if (h) destroy(h);
  return RS_OK;
}

}  // extern "C"
