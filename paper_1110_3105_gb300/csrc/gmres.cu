// Recursive skeletonization as a preconditioner (Sec. 6.4, multiple
// scattering): a system coupling p patches (scatterers),
//   sum_j A_ij sigma_j = f_i,   A_ii = the patch's own matrix I + w_i K_ii,
//                               A_ij = w_j K(patch i, patch j) (i != j),
// solved by GMRES with the block-diagonal preconditioner
// P^-1 = diag(A_11^-1, ..., A_pp^-1), each block applied by its patch's
// compressed inverse (one rs handle per patch).  The coupled matrix is
// applied densely from the coordinates (every pair of points, one warp per
// row); the paper applies it with an FMM, which is not part of this library.
//
// GMRES(m) with right preconditioning (Saad & Schultz 1986): the Arnoldi
// basis V of A P^-1 on the device, orthogonalised by classical Gram-Schmidt
// applied twice (one batched dot kernel and one update kernel per pass);
// the (m+1) x m Hessenberg matrix, its Givens rotations and the small
// triangular solve on the host (m <= 200 numbers); x = x0 + P^-1 V y at
// each restart.
#include <cmath>
#include <complex>
#include <vector>

#include "rs_internal.h"

namespace rs {

namespace {

constexpr int GM_NT = 256;

struct PatchPts {
  const double* x;     // points of every patch, caller order, per axis
  const double* y;
  const double* z;     // null in 2D
  const double* w;     // quadrature weight of each point (its patch's w)
  int64_t n;
};

template <class S> __device__ inline S scal_d(S a, double s) { return a * s; }
template <> __device__ inline c128 scal_d<c128>(c128 a, double s) { return c128(a.re * s, a.im * s); }
template <class S> __device__ inline S conj_s(S v) { return v; }
template <> __device__ inline c128 conj_s<c128>(c128 v) { return c128(v.re, -v.im); }
template <class S> __device__ inline S mul_s(S a, S b) { return a * b; }

// Green's function (no weight) between points i and j of the patch cloud.
template <class S> __device__ inline S green_pp(const KParams& kp, const PatchPts& p, int64_t i, int64_t j);
template <> __device__ inline double green_pp<double>(const KParams& kp, const PatchPts& p, int64_t i, int64_t j) {
  double dx = p.x[i] - p.x[j], dy = p.y[i] - p.y[j];
  double s = dx * dx + dy * dy;
  if (p.z) {
    const double dz = p.z[i] - p.z[j];
    s += dz * dz;
  }
  return green_real_s2(kp, s);
}
template <> __device__ inline c128 green_pp<c128>(const KParams& kp, const PatchPts& p, int64_t i, int64_t j) {
  double dx = p.x[i] - p.x[j], dy = p.y[i] - p.y[j];
  double s = dx * dx + dy * dy;
  if (p.z) {
    const double dz = p.z[i] - p.z[j];
    s += dz * dz;
  }
  return green_cplx(kp.kind, kp.kwave, sqrt(s));
}

// y = A x for the coupled matrix: y_i = x_i + sum_{j != i} w_j G(x_i, x_j) x_j.
template <class S>
__global__ void __launch_bounds__(GM_NT) k_coupled_apply(KParams kp, PatchPts p, const S* x, S* y) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (GM_NT / 32) + (threadIdx.x >> 5);
  if (i >= p.n) return;
  S acc = S(0.0);
  for (int64_t j = lane; j < p.n; j += 32)
    if (j != i) acc += scal_d(mul_s(green_pp<S>(kp, p, i, j), x[j]), p.w[j]);
  acc = warp_sum(acc);
  if (lane == 0) y[i] = x[i] + acc;
}

// h[c] = sum_i conj(V[:, c]) w (c < nc), one CTA per column.
template <class S>
__global__ void __launch_bounds__(GM_NT) k_dots(const S* V, int64_t ld, const S* w, int64_t n, S* h) {
  __shared__ S red[GM_NT / 32];
  const int c = blockIdx.x;
  S acc = S(0.0);
  for (int64_t i = threadIdx.x; i < n; i += GM_NT) acc += mul_s(conj_s(V[i + (int64_t)c * ld]), w[i]);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    S t = S(0.0);
    for (int q = 0; q < GM_NT / 32; ++q) t += red[q];
    h[c] = t;
  }
}

// w -= V[:, 0:nc] h  (or x += V y with sign = +1)
template <class S>
__global__ void k_update(const S* V, int64_t ld, const S* h, int nc, S* w, int64_t n, double sign) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    S acc = S(0.0);
    for (int c = 0; c < nc; ++c) acc += mul_s(V[i + (int64_t)c * ld], h[c]);
    w[i] += scal_d(acc, sign);
  }
}

template <class S>
__global__ void k_scale_copy(const S* src, S* dst, int64_t n, double f) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = scal_d(src[i], f);
}

template <class S>
__global__ void k_sub(const S* a, const S* b, S* out, int64_t n) {   // out = a - b
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] - b[i];
}

template <class S> struct HostT { using T = double; };
template <> struct HostT<c128> { using T = std::complex<double>; };
inline double cj(double v) { return v; }
inline std::complex<double> cj(std::complex<double> v) { return std::conj(v); }

template <class S>
int gmres_impl(int np, Handle* const* hs, const double* d_pts, const S* b, S* x, double tol, int max_it, int m,
               int precondition, int* its_out, double* relres_out, cudaStream_t st) {
  using H = typename HostT<S>::T;
  int64_t n = 0;
  std::vector<int64_t> seg(np + 1, 0);
  for (int i = 0; i < np; ++i) {
    seg[i] = n;
    n += hs[i]->N;
  }
  seg[np] = n;
  const int dim = hs[0]->dim;
  // device buffers: per-point weights, basis V (n x (m+1)), z, w, r, small vectors
  std::vector<void*> mem;
  auto alloc = [&](void** p, size_t bytes) -> int {
    if (cudaMallocAsync(p, std::max<size_t>(16, bytes), st) != cudaSuccess) {
      cudaGetLastError();
      return fail(RS_ERR_OOM, "rs_gmres_patches: workspace allocation failed");
    }
    mem.push_back(*p);
    return RS_OK;
  };
  int rc = RS_OK;
  double* wts = nullptr;
  S *V = nullptr, *z = nullptr, *w = nullptr, *r = nullptr, *hv = nullptr;
  do {
    if ((rc = alloc((void**)&wts, sizeof(double) * n)) != RS_OK) break;
    if ((rc = alloc((void**)&V, sizeof(S) * n * (m + 1))) != RS_OK) break;
    if ((rc = alloc((void**)&z, sizeof(S) * n)) != RS_OK) break;
    if ((rc = alloc((void**)&w, sizeof(S) * n)) != RS_OK) break;
    if ((rc = alloc((void**)&r, sizeof(S) * n)) != RS_OK) break;
    if ((rc = alloc((void**)&hv, sizeof(S) * (m + 1))) != RS_OK) break;
  } while (0);
  if (rc != RS_OK) {
    for (void* q : mem) cudaFreeAsync(q, st);
    return rc;
  }
  {
    std::vector<double> hw(n);
    for (int i = 0; i < np; ++i)
      for (int64_t q = seg[i]; q < seg[i + 1]; ++q) hw[q] = hs[i]->kp.w;
    cudaMemcpyAsync(wts, hw.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
  }
  PatchPts pp{d_pts, d_pts + n, dim == 3 ? d_pts + 2 * n : nullptr, wts, n};
  KParams kp = hs[0]->kp;
  kp.w = 1.0;
  const int rows_grid = (int)((n + GM_NT / 32 - 1) / (GM_NT / 32));
  const int vgrid = (int)std::min<int64_t>(4096, (n + 255) / 256);
  auto apply_A = [&](const S* in, S* out) -> int {
    k_coupled_apply<S><<<rows_grid, GM_NT, 0, st>>>(kp, pp, in, out);
    RS_CHECK_LAUNCH();
    return RS_OK;
  };
  auto apply_P = [&](const S* in, S* out) -> int {   // out = P^-1 in (block by block)
    if (!precondition) {
      RS_CUDA(cudaMemcpyAsync(out, in, sizeof(S) * n, cudaMemcpyDeviceToDevice, st));
      return RS_OK;
    }
    for (int i = 0; i < np; ++i)
      RS_TRY(solve_pers_device(hs[i], RS_PREC_FP64, in + seg[i], hs[i]->N, 1, out + seg[i], hs[i]->N, st));
    return RS_OK;
  };
  auto dots = [&](const S* Vb, int nc, const S* vec, std::vector<H>& out) -> int {
    k_dots<S><<<nc, GM_NT, 0, st>>>(Vb, n, vec, n, hv);
    RS_CHECK_LAUNCH();
    out.resize(nc);
    RS_CUDA(cudaMemcpyAsync(out.data(), hv, sizeof(S) * nc, cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaStreamSynchronize(st));
    return RS_OK;
  };
  auto nrm = [&](const S* vec, double* out) -> int {
    std::vector<H> t;
    RS_TRY(dots(vec, 1, vec, t));
    *out = std::sqrt(std::abs(t[0]));
    return RS_OK;
  };
  double bnorm = 0.0;
  int its = 0;
  double rel = 1.0;
  do {
    if ((rc = nrm(b, &bnorm)) != RS_OK) break;
    if (bnorm == 0.0) {
      RS_CUDA(cudaMemsetAsync(x, 0, sizeof(S) * n, st));
      rel = 0.0;
      break;
    }
    RS_CUDA(cudaMemsetAsync(x, 0, sizeof(S) * n, st));
    // restarts
    while (its < max_it) {
      // r = b - A x
      if ((rc = apply_A(x, w)) != RS_OK) break;
      k_sub<S><<<vgrid, 256, 0, st>>>(b, w, r, n);
      RS_CHECK_LAUNCH();
      double beta = 0.0;
      if ((rc = nrm(r, &beta)) != RS_OK) break;
      rel = beta / bnorm;
      if (rel <= tol) break;
      k_scale_copy<S><<<vgrid, 256, 0, st>>>(r, V, n, 1.0 / beta);
      RS_CHECK_LAUNCH();
      std::vector<std::vector<H>> Hm(m + 1, std::vector<H>(m, H(0.0)));
      std::vector<H> cs(m), sn(m), g(m + 1, H(0.0));
      g[0] = H(beta);
      int j = 0;
      for (; j < m && its < max_it; ++j) {
        ++its;
        S* vj = V + (int64_t)j * n;
        if ((rc = apply_P(vj, z)) != RS_OK) break;
        if ((rc = apply_A(z, w)) != RS_OK) break;
        std::vector<H> h1, h2;
        for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
          std::vector<H>& hh = pass ? h2 : h1;
          if ((rc = dots(V, j + 1, w, hh)) != RS_OK) break;
          RS_CUDA(cudaMemcpyAsync(hv, hh.data(), sizeof(S) * (j + 1), cudaMemcpyHostToDevice, st));
          k_update<S><<<vgrid, 256, 0, st>>>(V, n, hv, j + 1, w, n, -1.0);
          RS_CHECK_LAUNCH();
        }
        if (rc != RS_OK) break;
        for (int i = 0; i <= j; ++i) Hm[i][j] = h1[i] + h2[i];
        double hn = 0.0;
        if ((rc = nrm(w, &hn)) != RS_OK) break;
        Hm[j + 1][j] = H(hn);
        if (hn > 0.0) {
          k_scale_copy<S><<<vgrid, 256, 0, st>>>(w, V + (int64_t)(j + 1) * n, n, 1.0 / hn);
          RS_CHECK_LAUNCH();
        }
        // Givens rotations on column j of the Hessenberg matrix: (c real, s)
        // with [c s; -conj(s) c] [a; b] = [nu a / |a|; 0]
        for (int i = 0; i < j; ++i) {
          const H t = cs[i] * Hm[i][j] + sn[i] * Hm[i + 1][j];
          Hm[i + 1][j] = -cj(sn[i]) * Hm[i][j] + cs[i] * Hm[i + 1][j];
          Hm[i][j] = t;
        }
        {
          const H a = Hm[j][j], bb = Hm[j + 1][j];
          const double aa = std::abs(a), nu = std::sqrt(aa * aa + std::abs(bb) * std::abs(bb));
          if (nu == 0.0) {
            cs[j] = H(1.0);
            sn[j] = H(0.0);
          } else if (aa == 0.0) {
            cs[j] = H(0.0);
            sn[j] = H(1.0);
          } else {
            cs[j] = H(aa / nu);
            sn[j] = (a / aa) * cj(bb) / nu;
          }
        }
        Hm[j][j] = cs[j] * Hm[j][j] + sn[j] * Hm[j + 1][j];
        Hm[j + 1][j] = H(0.0);
        g[j + 1] = -cj(sn[j]) * g[j];
        g[j] = cs[j] * g[j];
        rel = std::abs(g[j + 1]) / bnorm;
        if (rel <= tol || hn == 0.0) {
          ++j;
          break;
        }
      }
      if (rc != RS_OK) break;
      // y from the triangular system, x += P^-1 (V y)
      std::vector<H> y(j, H(0.0));
      for (int i = j - 1; i >= 0; --i) {
        H s = g[i];
        for (int q = i + 1; q < j; ++q) s -= Hm[i][q] * y[q];
        y[i] = Hm[i][i] == H(0.0) ? H(0.0) : s / Hm[i][i];
      }
      RS_CUDA(cudaMemcpyAsync(hv, y.data(), sizeof(S) * j, cudaMemcpyHostToDevice, st));
      RS_CUDA(cudaMemsetAsync(w, 0, sizeof(S) * n, st));
      k_update<S><<<vgrid, 256, 0, st>>>(V, n, hv, j, w, n, 1.0);
      RS_CHECK_LAUNCH();
      if ((rc = apply_P(w, z)) != RS_OK) break;
      {   // x += z
        const S one = S(1.0);
        RS_CUDA(cudaMemcpyAsync(hv, &one, sizeof(S), cudaMemcpyHostToDevice, st));
        k_update<S><<<vgrid, 256, 0, st>>>(z, n, hv, 1, x, n, 1.0);
        RS_CHECK_LAUNCH();
      }
      if (rel <= tol) {   // the true residual decides (the loop head recomputes it)
        if ((rc = apply_A(x, w)) != RS_OK) break;
        k_sub<S><<<vgrid, 256, 0, st>>>(b, w, r, n);
        RS_CHECK_LAUNCH();
        double rn = 0.0;
        if ((rc = nrm(r, &rn)) != RS_OK) break;
        rel = rn / bnorm;
        if (rel <= tol) break;
      }
    }
  } while (0);
  cudaError_t e = cudaStreamSynchronize(st);
  for (void* q : mem) cudaFreeAsync(q, st);
  if (rc == RS_OK && e != cudaSuccess) rc = fail(RS_ERR_CUDA, "rs_gmres_patches: %s", cudaGetErrorString(e));
  for (int i = 0; i < np && rc == RS_OK; ++i) rc = pers_check(hs[i]);
  if (its_out) *its_out = its;
  if (relres_out) *relres_out = rel;
  return rc;
}

}  // namespace

int gmres_patches_device(int np, Handle* const* hs, const double* d_pts, const void* b, void* x, double tol,
                         int max_it, int restart, int precondition, int* its_out, double* relres_out,
                         cudaStream_t st) {
  if (hs[0]->cplx)
    return gmres_impl<c128>(np, hs, d_pts, (const c128*)b, (c128*)x, tol, max_it, restart, precondition, its_out,
                            relres_out, st);
  return gmres_impl<double>(np, hs, d_pts, (const double*)b, (double*)x, tol, max_it, restart, precondition, its_out,
                            relres_out, st);
}

}  // namespace rs
