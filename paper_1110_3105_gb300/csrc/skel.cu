// Per-level skeletonization and factorization (the build's hot path).
//
// For every box of one tree depth, one CTA:
//   k_id      fills the proxy-compressed matrix
//               M = [ w G(near, I) ; w G(proxy, I) (; w 1) ]      (Sec. 3.2)
//             (near = active points of the colleague boxes, proxy surface as
//             in the header rs.h describes) and computes its interpolative
//             decomposition (Sec. 2.2, Def. 2.3) by Householder QR with column
//             pivoting: pivot = largest trailing column norm (norms recomputed
//             every step, lowest index on ties, warp-level argmax), rank k =
//             first j with |R_jj| <= eps |R_00|, T = R11^-1 R12.
//   k_factor  assembles the diagonal block D (leaf: A(I, I); above: the
//             children's Lambda on the diagonal, w G between skeletons of
//             different children -- S^(l-1) regrouped plus Lambda^(l-1), eqs.
//             sparse-embedding / multilevel-embedding) and eliminates it
//             (eq. compressed-inverse) with P = [I T] Pi, L = P^T, R = P:
//               X = D^-1 P^T,  Lambda = (P X)^-1,  calL = X Lambda,
//               calR = Lambda X^T (D symmetric: P D^-1 = X^T),
//               calD = D^-1 - calL X^T.
// Everything is double (complex double for Helmholtz); the rank decision and
// every LU stay in FP64.  Dense inverses use Gauss-Jordan elimination with
// partial pivoting on [D | I].
#include <algorithm>
#include <cmath>
#include <vector>

#include <cooperative_groups.h>
#include <cuda/atomic>
#include <type_traits>

#include "rs_internal.h"

namespace rs {

namespace {

constexpr int ID_NT = 256;
constexpr int FA_NT = 256;
constexpr int FA_SM_NT = 128;

// Load through L2 (data another CTA of the same launch may have written).
template <class S> __device__ inline S ldcg_s(const S* p) { return __ldcg(p); }
template <> __device__ inline c128 ldcg_s<c128>(const c128* p) {
  const double2 t = __ldcg(reinterpret_cast<const double2*>(p));
  return c128(t.x, t.y);
}

template <class S> __device__ inline S scal(S a, double s);
template <> __device__ inline double scal<double>(double a, double s) { return a * s; }
template <> __device__ inline c128 scal<c128>(c128 a, double s) { return c128(a.re * s, a.im * s); }

struct Geo {
  double lower[3];
  double side;      // box side at this depth
  int dim;
  int nproxy;
  double ratio;
  int constrow;     // 1: append a constant row (2D Laplace with |log rho| < 0.1)
};

// Coordinates of proxy point j of a box with the given integer coordinates.
__device__ inline void proxy_point(const Geo& g, const int* coords, int j, double* out) {
  double c[3];
  for (int d = 0; d < g.dim; ++d) c[d] = g.lower[d] + ((double)coords[d] + 0.5) * g.side;
  if (g.dim == 2) {
    double rho = g.ratio * (0.70710678118654752440) * g.side;
    double th = 2.0 * M_PI * (double)j / (double)g.nproxy;
    out[0] = c[0] + rho * cos(th);
    out[1] = c[1] + rho * sin(th);
    out[2] = 0.0;
    return;
  }
  int gg = (int)lrint(sqrt((double)g.nproxy / 6.0));
  double h = g.ratio * g.side * 0.5;
  int face = j / (gg * gg), rem = j % (gg * gg);
  int ia = rem / gg, ib = rem % gg;
  int axis = face / 2;
  double sign = (face % 2) ? 1.0 : -1.0;
  double ua = -h + (2.0 * ia + 1.0) * h / gg;
  double ub = -h + (2.0 * ib + 1.0) * h / gg;
  double p[3];
  p[axis] = sign * h;
  int o0 = axis == 0 ? 1 : 0;
  int o1 = axis == 2 ? 1 : 2;
  p[o0] = ua;
  p[o1] = ub;
  for (int d = 0; d < 3; ++d) out[d] = c[d] + p[d];
}

__device__ inline double dist2_to(const Pts& p, int i, const double* q) {
  double dx = p.x[i] - q[0], dy = p.y[i] - q[1];
  double s = dx * dx + dy * dy;
  if (p.z) { double dz = p.z[i] - q[2]; s += dz * dz; }
  return s;
}

// Column-pivoted Householder QR of M (m x n, column-major, leading dim ld),
// stopped at relative precision eps but not before kmin steps (unless the
// trailing matrix is exactly zero).  On return piv holds the column order,
// M[0:k, 0:n] the triangular factor; returns k.
//
// The trailing column norms that choose the pivots are downdated after each
// step (|R_jc|^2 subtracted) and recomputed from the column once the
// downdate has cancelled more than a factor 1.5e-8 of the last exact value
// (the safeguard of LAPACK's xGEQP3, Drmac & Bujanovic 2008), so a step costs
// two FP64 passes over the trailing matrix instead of three.  The pivot's own
// norm, which sets R_jj, the reflector and the stopping test, is always
// recomputed exactly.  nrm holds 2 n doubles (current | last exact).
template <class S, int NT>
__device__ int cpqr(S* M, int m, int n, int ld, double eps, int* piv, double* nrm, S* u, int kmin = 0) {
  __shared__ int s_p, s_stop;
  __shared__ double s_rjj, s_r00;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NT / 32;
  constexpr int QG = 8, QCW = 32 / QG;
  const int gl = lane & (QG - 1), grp = lane / QG;
  constexpr double kTol = 1.49e-8;   // sqrt of the double unit roundoff
  double* nref = nrm + n;
  for (int c = tid; c < n; c += NT) piv[c] = c;
  const int kmax = min(m, n);
  for (int c = warp; c < n; c += NW) {
    const S* col = M + (size_t)c * ld;
    double s = 0.0;
    for (int r = lane; r < m; r += 32) s += abs2(col[r]);
    s = warp_sum(s);
    if (lane == 0) nrm[c] = nref[c] = s;
  }
  __syncthreads();
  int j = 0;
  for (; j < kmax; ++j) {
    if (warp == 0) {
      double best = -1.0;
      int bi = n;
      for (int c = j + lane; c < n; c += 32) {
        double v = nrm[c];
        if (v > best) { best = v; bi = c; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) s_p = bi;
    }
    __syncthreads();
    const int p = s_p;
    if (p != j) {
      for (int r = tid; r < m; r += NT) {
        S t = M[r + (size_t)j * ld];
        M[r + (size_t)j * ld] = M[r + (size_t)p * ld];
        M[r + (size_t)p * ld] = t;
      }
      if (tid == 0) {
        int t = piv[j]; piv[j] = piv[p]; piv[p] = t;
        double a = nrm[j]; nrm[j] = nrm[p]; nrm[p] = a;
        a = nref[j]; nref[j] = nref[p]; nref[p] = a;
      }
    }
    __syncthreads();
    if (warp == 0) {   // exact norm of the pivot column over rows j..m-1
      const S* col = M + (size_t)j * ld;
      double s = 0.0;
      for (int r = j + lane; r < m; r += 32) s += abs2(col[r]);
      s = warp_sum(s);
      if (lane == 0) {
        const double rjj = sqrt(s);
        int stop = 0;
        if (j == 0) {
          s_r00 = rjj;
          if (!(rjj > 0.0)) stop = 1;
        } else if (rjj <= eps * s_r00 && (j >= kmin || !(rjj > 0.0))) {
          stop = 1;
        }
        s_rjj = rjj;
        s_stop = stop;
      }
    }
    __syncthreads();
    if (s_stop) break;
    const double rjj = s_rjj;
    // Householder reflector H = I - f u u^H mapping column j onto beta e_1,
    // beta = -phase(alpha) ||x||, u = x - beta e_1, f = 2 / (u^H u).
    const S alpha = M[j + (size_t)j * ld];
    const double aa = sqrt(abs2(alpha));
    const S phase = aa > 0.0 ? scal(alpha, 1.0 / aa) : S(1.0);
    const S beta = scal(phase, -rjj);
    for (int r = j + tid; r < m; r += NT) u[r - j] = (r == j) ? alpha - beta : M[r + (size_t)j * ld];
    const double f = 1.0 / (rjj * (rjj + aa));
    __syncthreads();
    // Trailing columns: a group of QG lanes per column (QCW columns per warp),
    // each lane a strided share of the rows, so the dot product's reduction
    // is log2(QG) shuffles shared by QCW columns.
    for (int cb = j + 1 + warp * QCW; cb < n; cb += NW * QCW) {
      const int c = cb + grp;
      const bool act = c < n;
      S* col = M + (size_t)(act ? c : j) * ld;
      S s = S(0.0);
      if (act)
        for (int r = j + gl; r < m; r += QG) s += conj_(u[r - j]) * col[r];
      s = group_sum<QG>(s);
      const S fs = scal(s, f);
      if (act)
        for (int r = j + gl; r < m; r += QG) col[r] = col[r] - u[r - j] * fs;
      __syncwarp();
      int again = 0;
      if (act && gl == 0) {   // row j of the column was updated by this lane
        const double left = nrm[c] - abs2(col[j]);
        if (left <= kTol * nref[c]) again = 1;
        else nrm[c] = left;
      }
      again = __shfl_sync(0xffffffffu, again, grp * QG);
      if (__any_sync(0xffffffffu, again)) {   // too much cancelled: recompute
        double s2 = 0.0;
        if (again)
          for (int r = j + 1 + gl; r < m; r += QG) s2 += abs2(col[r]);
        s2 = group_sum<QG>(s2);
        if (again && gl == 0) nrm[c] = nref[c] = s2;
      }
    }
    if (tid == 0) M[j + (size_t)j * ld] = beta;
    __syncthreads();
  }
  return j;
}

// T = R11^-1 R12 in place in M[0:k, k:n]; one warp per column.
template <class S, int NT>
__device__ void back_substitute(S* M, int k, int n, int ld) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  for (int c = k + warp; c < n; c += NW) {
    S* col = M + (size_t)c * ld;
    for (int i = k - 1; i >= 0; --i) {
      S ti = S(0.0);
      if (lane == 0) {
        ti = col[i] / M[i + (size_t)i * ld];
        col[i] = ti;
      }
      ti = shfl(ti, 0);
      for (int r = lane; r < i; r += 32) col[r] -= M[r + (size_t)i * ld] * ti;
      __syncwarp();
    }
  }
}


// ------------------------------------------------ double-float pivoted QR
// The real-kernel ID runs its QR on the FP32 pipes in double-float
// arithmetic (hi + lo floats, about 48 significant bits; see rs_common.cuh):
// on GB300 an FP64 FMA costs as much issue as 64 FP32 FMAs, and the ~12 FP32
// instructions of a double-float multiply-add still come out five times
// cheaper.  A backward error near m * 2^-48 ~ 1e-12 is far below the
// skeletonization tolerance (eps >= 1e-10 in every configuration), so ranks,
// pivots (up to near-ties) and T agree with the FP64 factorization.  The
// O(n) scalars of a step (norms, R_jj, the reflector's alpha, beta and f)
// stay in FP64; only the O(m n) passes run in double-float.
__device__ __forceinline__ double df_to_d(dfloat v) { return __dadd_rn(f32_to_f64(v.hi), f32_to_f64(v.lo)); }
__device__ __forceinline__ dfloat df_warp_sum(dfloat v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = v + dfloat(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
  return v;
}
// s += a * b, renormalized (|lo| <= ulp(hi) / 2) for values that are updated
// again and again.
__device__ __forceinline__ void df_fma_n(dfloat& s, dfloat a, dfloat b) {
  df_fma(s, a, b);
  s = df_renorm(s);
}

template <int NT>
__device__ int cpqr_df(dfloat* M, int m, int n, int ld, double eps, int* piv, double* nrm, dfloat* u,
                       int kmin = 0) {
  __shared__ int s_p, s_stop;
  __shared__ double s_rjj, s_r00;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NT / 32;
  constexpr double kTol = 1.49e-8;
  double* nref = nrm + n;
  for (int c = tid; c < n; c += NT) piv[c] = c;
  const int kmax = min(m, n);
  for (int c = warp; c < n; c += NW) {
    const dfloat* col = M + (size_t)c * ld;
    dfloat s(0.0f, 0.0f);
    for (int r = lane; r < m; r += 32) df_fma(s, col[r], col[r]);
    s = df_warp_sum(s);
    if (lane == 0) nrm[c] = nref[c] = df_to_d(s);
  }
  __syncthreads();
  int j = 0;
  for (; j < kmax; ++j) {
    if (warp == 0) {
      double best = -1.0;
      int bi = n;
      for (int c = j + lane; c < n; c += 32) {
        double v = nrm[c];
        if (v > best) { best = v; bi = c; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) s_p = bi;
    }
    __syncthreads();
    const int p = s_p;
    if (p != j) {
      for (int r = tid; r < m; r += NT) {
        dfloat t = M[r + (size_t)j * ld];
        M[r + (size_t)j * ld] = M[r + (size_t)p * ld];
        M[r + (size_t)p * ld] = t;
      }
      if (tid == 0) {
        int t = piv[j]; piv[j] = piv[p]; piv[p] = t;
        double a = nrm[j]; nrm[j] = nrm[p]; nrm[p] = a;
        a = nref[j]; nref[j] = nref[p]; nref[p] = a;
      }
    }
    __syncthreads();
    if (warp == 0) {   // norm of the pivot column over rows j..m-1
      const dfloat* col = M + (size_t)j * ld;
      dfloat s(0.0f, 0.0f);
      for (int r = j + lane; r < m; r += 32) df_fma(s, col[r], col[r]);
      s = df_warp_sum(s);
      if (lane == 0) {
        const double rjj = sqrt(df_to_d(s));
        int stop = 0;
        if (j == 0) {
          s_r00 = rjj;
          if (!(rjj > 0.0)) stop = 1;
        } else if (rjj <= eps * s_r00 && (j >= kmin || !(rjj > 0.0))) {
          stop = 1;
        }
        s_rjj = rjj;
        s_stop = stop;
      }
    }
    __syncthreads();
    if (s_stop) break;
    const double rjj = s_rjj;
    // Householder reflector H = I - f u u^T mapping column j onto beta e_1
    const double alpha = df_to_d(M[j + (size_t)j * ld]);
    const double aa = fabs(alpha);
    const double beta = alpha < 0.0 ? rjj : -rjj;
    for (int r = j + tid; r < m; r += NT) u[r - j] = (r == j) ? f64_to_df(alpha - beta) : M[r + (size_t)j * ld];
    const double f = 1.0 / (rjj * (rjj + aa));
    __syncthreads();
    for (int c = j + 1 + warp; c < n; c += NW) {
      dfloat* col = M + (size_t)c * ld;
      dfloat s(0.0f, 0.0f);
      for (int r = j + lane; r < m; r += 32) df_fma(s, u[r - j], col[r]);
      s = df_warp_sum(s);
      const dfloat nfs = f64_to_df(-f * df_to_d(s));
      for (int r = j + lane; r < m; r += 32) df_fma_n(col[r], u[r - j], nfs);
      __syncwarp();
      int again = 0;
      if (lane == 0) {
        const double rj = df_to_d(col[j]);
        const double left = nrm[c] - rj * rj;
        if (left <= kTol * nref[c]) again = 1;
        else nrm[c] = left;
      }
      if (__shfl_sync(0xffffffffu, again, 0)) {   // too much cancelled: recompute
        dfloat s2(0.0f, 0.0f);
        for (int r = j + 1 + lane; r < m; r += 32) df_fma(s2, col[r], col[r]);
        s2 = df_warp_sum(s2);
        if (lane == 0) nrm[c] = nref[c] = df_to_d(s2);
      }
    }
    if (tid == 0) M[j + (size_t)j * ld] = f64_to_df(beta);
    __syncthreads();
  }
  return j;
}

// T = R11^-1 R12 in place in M[0:k, k:n] (double-float); one warp per column.
template <int NT>
__device__ void back_substitute_df(dfloat* M, int k, int n, int ld) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  for (int c = k + warp; c < n; c += NW) {
    dfloat* col = M + (size_t)c * ld;
    for (int i = k - 1; i >= 0; --i) {
      double ti = 0.0;
      if (lane == 0) {
        ti = df_to_d(col[i]) / df_to_d(M[i + (size_t)i * ld]);
        col[i] = f64_to_df(ti);
      }
      ti = __shfl_sync(0xffffffffu, ti, 0);
      const dfloat nti = f64_to_df(-ti);
      for (int r = lane; r < i; r += 32) df_fma_n(col[r], M[r + (size_t)i * ld], nti);
      __syncwarp();
    }
  }
}

struct IdArgs {
  KParams kp;
  Pts pts;
  Geo geo;
  double eps;
  const int* n;          // per box active size
  const int64_t* off;    // per box active offset
  const int* act;        // active point ids
  const int* ncoll;
  const int* coll;
  const int* coords;
  const int* mrows;      // per box total rows
  const int64_t* moff;   // per box workspace offset (global path)
  const int64_t* toff;
  int* kout;
  int* lperm;
  // two-sided IDs (non-symmetric kernels): act_near = the colleagues' point
  // ids that make the near-field rows (the row active set for the column
  // ID, the column active set for the row ID; = act for symmetric kernels);
  // row_side = 1: the transposed row ID (entries K(box point, near point),
  // proxy rows from single-layer charges on the proxy circle, a constant
  // row); kmin: per-box minimum rank (null: none)
  const int* act_near;
  int row_side;
  const int* kmin;
  // near-field blocks shared by colleague pairs (k_near_pairs): for box b's
  // colleague slot s, the block G(I_j, I_b) starts at pair_base[27 b + s] of
  // pairs, stored for the lower-numbered box of the pair (n_j x n_b
  // column-major when j > b, its transpose when j < b); null: evaluate
  const int64_t* pair_base;
  const void* pairs;
  int smem_path;         // 1: M in shared memory
  int qr_df;             // 1: double-float QR (real kernels, rs_id_arith)
  // randomized ID (Sec. 2.2): with sketch_p > 0 a box whose m exceeds
  // n + sketch_p is compressed through its sample Omega M (n + sketch_p
  // rows); Omega(i, r) = sketch[i + r * SKETCH_STRIDE]
  const double* sketch;
  int sketch_p;
  int mmax, nmax;
  int64_t mnmax;         // max over boxes of m n (the shared M, leading dimension m)
};

constexpr int SKETCH_STRIDE = 1024;   // rows of the sketch table (the largest sample)
constexpr int SKETCH_STREAM = 77;

// splitmix64 (Steele, Lea & Flood 2014) of one 64-bit counter.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = (x + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double uniform01(uint64_t seed, uint64_t stream, uint64_t idx) {
  const uint64_t base = (seed * 0x100000001B3ull) ^ (stream << 40);
  return ((double)(splitmix64(idx + base) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

// The sketch table: entry e = r * SKETCH_STRIDE + i is element e of the
// normal stream of the seed (Box-Muller on pairs of splitmix64 uniforms:
// element 2p = rad cos(2 pi u2), 2p + 1 = rad sin(2 pi u2), rad =
// sqrt(-2 log u1), u1 and u2 the p-th uniforms of streams 2 s and 2 s + 1).
__global__ void k_sketch_table(uint64_t seed, int64_t count, double* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t pi = (uint64_t)e >> 1;
    const double u1 = uniform01(seed, 2 * SKETCH_STREAM, pi), u2 = uniform01(seed, 2 * SKETCH_STREAM + 1, pi);
    const double rad = sqrt(-2.0 * log(u1));
    const double ang = 2.0 * M_PI * u2;
    out[e] = (e & 1) ? rad * sin(ang) : rad * cos(ang);
  }
}

template <class S, int NT>
__global__ void __launch_bounds__(NT) k_id(IdArgs a, S* Mws, S* Tpool) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int cstart[28];
  const int b = blockIdx.x;
  const int n = a.n[b];
  const int m = a.mrows[b];
  const int64_t off = a.off[b];
  // shared layout: [M (smem path)] | u[mmax] | nrm[2 nmax] | proxy xyz[3 nproxy] | rbase[mmax] (int64) |
  // piv[nmax] | rowid[mmax] | rstride[mmax]
  S* Ms = reinterpret_cast<S*>(smem);
  size_t msz = a.smem_path ? (size_t)a.mnmax : 0;
  S* u = Ms + msz;
  double* nrm = reinterpret_cast<double*>(u + a.mmax);
  double* pxy = nrm + 2 * a.nmax;
  int64_t* rbase = reinterpret_cast<int64_t*>(pxy + 3 * a.geo.nproxy);
  int* piv = reinterpret_cast<int*>(rbase + a.mmax);
  int* rowid = piv + a.nmax;
  int* rstride = rowid + a.mmax;
  const S* pairs = reinterpret_cast<const S*>(a.pairs);
  S* M = a.smem_path ? Ms : Mws + a.moff[b];
  const int ld = m;
  const int nc = a.ncoll[b];

  // near-field rows: colleagues' active sets in ascending box order
  if (threadIdx.x == 0) {
    int r = 0;
    for (int j = 0; j < nc; ++j) {
      cstart[j] = r;
      r += a.n[a.coll[b * 27 + j]];
    }
    cstart[nc] = r;
  }
  __syncthreads();
  const int nnear = cstart[nc];
  for (int r = threadIdx.x; r < nnear; r += NT) {
    int j = 0;
    while (cstart[j + 1] <= r) ++j;
    int c = a.coll[b * 27 + j];
    const int q = r - cstart[j];
    rowid[r] = a.act_near[a.off[c] + q];
    rstride[r] = 0;   // 0: evaluate the entry
    if (pairs) {      // row q of colleague c in the shared block of the pair
      const int64_t base = a.pair_base[b * 27 + j];
      if (base >= 0) {
        if (c > b) { rbase[r] = base + q; rstride[r] = a.n[c]; }
        else { rbase[r] = base + (int64_t)q * n; rstride[r] = 1; }
      }
    }
  }
  __syncthreads();

  // proxy surface of this box, once
  const int* bc = a.coords + (size_t)b * a.geo.dim;
  for (int j = threadIdx.x; j < a.geo.nproxy; j += NT) proxy_point(a.geo, bc, j, pxy + 3 * j);
  __syncthreads();
  // fill M column-major: rows = near | proxy | (constant)
  const int64_t total = (int64_t)m * n;
  for (int64_t e = threadIdx.x; e < total; e += NT) {
    int r = (int)(e % m), c = (int)(e / m);
    int pc = a.act[off + c];
    S v;
    if (r < nnear) {
      v = rstride[r] ? pairs[rbase[r] + (int64_t)c * rstride[r]]
          : a.row_side ? offdiag_entry<S>(a.kp, a.pts, pc, rowid[r]) : offdiag_entry<S>(a.kp, a.pts, rowid[r], pc);
    } else if (r < nnear + a.geo.nproxy) {
      const double* pp = pxy + 3 * (r - nnear);
      if (a.kp.kind != RS_LAPLACE2D_DL) v = green_at_s2<S>(a.kp, dist2_to(a.pts, pc, pp));
      else if (a.row_side) v = S(-a.kp.w * (0.25 / M_PI) * log_tab(a.kp.logtab, dist2_to(a.pts, pc, pp)));
      else v = S(a.kp.w * dlayer_at(a.pts, pp[0], pp[1], pc));
    } else {   // the constant row (2D Laplace near radius 1; the double layer's row ID)
      v = (a.kp.kind != RS_LAPLACE2D_DL || a.row_side) ? S(a.kp.w) : S(0.0);
    }
    if constexpr (std::is_same<S, double>::value)
      if (a.qr_df) {
        reinterpret_cast<dfloat*>(M)[r + (size_t)c * ld] = f64_to_df(v);
        continue;
      }
    M[r + (size_t)c * ld] = v;
  }
  __syncthreads();

  // randomized ID: the pivoted QR of the sample Omega M (l = n + p rows)
  // instead of M; the sample overwrites M's first l rows column by column
  int mq = m;
  if (a.sketch_p > 0 && m > n + a.sketch_p) {
    const int l = n + a.sketch_p;
    for (int c = 0; c < n; ++c) {
      const S* col = M + (size_t)c * ld;
      for (int i = threadIdx.x; i < l; i += NT) {
        S acc = S(0.0);
        for (int r = 0; r < m; ++r) acc += scal(col[r], a.sketch[i + (size_t)r * SKETCH_STRIDE]);
        u[i] = acc;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < l; i += NT) M[i + (size_t)c * ld] = u[i];
      __syncthreads();
    }
    mq = l;
  }

  S* T = Tpool + a.toff[b];
  int k;
  bool done = false;
  if constexpr (std::is_same<S, double>::value)
    if (a.qr_df) {   // the fill stored the matrix as double-float
      dfloat* Md = reinterpret_cast<dfloat*>(M);
      k = cpqr_df<NT>(Md, m, n, ld, a.eps, piv, nrm, reinterpret_cast<dfloat*>(u), a.kmin ? a.kmin[b] : 0);
      __syncthreads();
      back_substitute_df<NT>(Md, k, n, ld);
      __syncthreads();
      const int nr = n - k;
      for (int e = threadIdx.x; e < k * nr; e += NT) {
        int r = e % k, c = e / k;
        T[r + (size_t)c * k] = df_to_d(Md[r + (size_t)(k + c) * ld]);
      }
      done = true;
    }
  if (!done) {
    k = cpqr<S, NT>(M, mq, n, ld, a.eps, piv, nrm, u, a.kmin ? a.kmin[b] : 0);
    __syncthreads();
    back_substitute<S, NT>(M, k, n, ld);
    __syncthreads();
    const int nr = n - k;
    for (int e = threadIdx.x; e < k * nr; e += NT) {
      int r = e % k, c = e / k;
      T[r + (size_t)c * k] = M[r + (size_t)(k + c) * ld];
    }
  }
  for (int c = threadIdx.x; c < n; c += NT) a.lperm[off + c] = piv[c];
  if (threadIdx.x == 0) a.kout[b] = k;
}

// Near-field kernel blocks of one depth, once per colleague pair (i, j), i < j:
// G(I_j, I_i) (n_j x n_i, column-major) at base[p]; the two boxes read it
// directly and transposed (k_id), halving the near-field evaluations.
template <class S>
__global__ void k_near_pairs(KParams kp, Pts pts, const int* n, const int64_t* off, const int* act, const int* pi,
                             const int* pj, const int64_t* base, S* out) {
  const int p = blockIdx.x;
  const int i = pi[p], j = pj[p];
  const int ni = n[i], nj = n[j];
  const int* ai = act + off[i];
  const int* aj = act + off[j];
  S* o = out + base[p];
  for (int e = threadIdx.x; e < ni * nj; e += blockDim.x) {
    const int a = e % nj, c = e / nj;
    o[e] = offdiag_entry<S>(kp, pts, aj[a], ai[c]);
  }
}

// ---------------------------------------------------------- big-box ID
// For boxes whose compressed matrix does not fit one CTA's shared memory:
// the same pivoted QR, with one launch per pivot step and each CTA owning 32
// physical columns of one box.  Column exchanges only permute a
// position -> column map (double-buffered across launches); the trailing
// norms, the rank and R_00 live in global memory, so every CTA of a box takes
// the same pivot and stop decision from the previous launch's values.
struct BigId {
  const int* m;          // rows per box
  const int* n;
  const int64_t* moff;   // M offset per box (scalars)
  const int64_t* noff;   // offset of per-column arrays per box
  double* nrm;           // trailing column norms^2 (per physical column), two parities
  int64_t ntot;          // entries of one parity
  int* map0;             // position -> physical column, parity 0
  int* map1;             // parity 1
  double* r00;           // per box
  int* kk;               // per box rank (starts at min(m, n))
  void* rdiag;           // R_jj per position (scalars, same offsets as nrm)
};

constexpr int BI_NT = 128;
constexpr int BI_CB = 8;

// Grid-wide barrier of a cooperative launch (every CTA resident): CTAs add
// to a monotonic arrival counter and wait for gridDim.x arrivals per step.
// Waits are bounded: past BAR_SPIN polls a CTA raises *flag and leaves, and
// every waiter also polls the flag, so a stuck grid drains instead of hanging.
constexpr int BAR_SPIN = 1 << 22;
struct GridBar {
  unsigned int* count;
  int* flag;
};
__device__ inline bool grid_sync(GridBar gb, unsigned int target) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(gb.count, 1u);
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(*gb.count);
    int ok = 1, spins = 0;
    while (cnt.load(cuda::memory_order_acquire) < target) {
      if (*(volatile int*)gb.flag || ++spins > BAR_SPIN) {
        atomicExch(gb.flag, 1);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <class S>
__global__ void __launch_bounds__(BI_NT) k_bbid_fill(IdArgs a, BigId g, S* Mws, int maxn) {
  __shared__ int cstart[28];
  __shared__ double pxy[3 * 256];
  const int b = blockIdx.x / maxn, c = blockIdx.x % maxn;
  const int n = a.n[b];
  if (c >= n) return;
  const int m = g.m[b];
  const int64_t off = a.off[b];
  const int nc = a.ncoll[b];
  if (threadIdx.x == 0) {
    int r = 0;
    for (int j = 0; j < nc; ++j) {
      cstart[j] = r;
      r += a.n[a.coll[b * 27 + j]];
    }
    cstart[nc] = r;
  }
  const int* bc = a.coords + (size_t)b * a.geo.dim;
  for (int j = threadIdx.x; j < a.geo.nproxy; j += BI_NT) proxy_point(a.geo, bc, j, pxy + 3 * j);
  __syncthreads();
  const int nnear = cstart[nc];
  const int pc = a.act[off + c];
  S* col = Mws + g.moff[b] + (size_t)c * m;
  double s2 = 0.0;
  for (int r = threadIdx.x; r < m; r += BI_NT) {
    S v;
    if (r < nnear) {
      int j = 0;
      while (cstart[j + 1] <= r) ++j;
      int cc = a.coll[b * 27 + j];
      v = offdiag_entry<S>(a.kp, a.pts, a.act[a.off[cc] + (r - cstart[j])], pc);
    } else if (r < nnear + a.geo.nproxy) {
      v = green_at_s2<S>(a.kp, dist2_to(a.pts, pc, pxy + 3 * (r - nnear)));
    } else {
      v = S(a.kp.w);
    }
    col[r] = v;
    s2 += abs2(v);
  }
  __shared__ double red[BI_NT];
  red[threadIdx.x] = s2;
  __syncthreads();
  for (int o = BI_NT / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    g.nrm[g.noff[b] + c] = red[0];
    g.map0[g.noff[b] + c] = c;
    if (c == 0) g.kk[b] = min(m, n);
  }
}

// One pivot step; each CTA owns CB physical columns of one box.  With Ms
// (cooperative launch) the CTA's own columns are also kept in shared memory,
// [CB][m]: read from there, written to both.
template <class S, int CB>
__device__ void bbid_body(const IdArgs& a, const BigId& g, S* Mws, int j, int ncb, int* lperm, S* Ms) {
  extern __shared__ __align__(16) unsigned char bi_smem[];
  S* u = reinterpret_cast<S*>(bi_smem);                  // mmax entries
  int* mp = reinterpret_cast<int*>(u + a.mmax);          // nmax entries
  __shared__ int s_p, s_stop;
  __shared__ double s_rjj, s_r00;
  __shared__ int s_kk;
  const int b = blockIdx.x / ncb, cb = blockIdx.x % ncb;
  const int n = a.n[b], m = g.m[b];
  const int kmax = min(m, n);
  // Data written by other CTAs during the step loop (maps, norms, the pivot
  // column, rank and R_00) is read through L2 (__ldcg).  The rank is read
  // once per CTA so the early exit below is uniform.
  if (threadIdx.x == 0) s_kk = __ldcg(g.kk + b);
  __syncthreads();
  if (j >= kmax || s_kk < kmax) return;   // past the rank or already stopped
  if (cb * CB >= n) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t no = g.noff[b];
  const int* map_in = (j & 1) ? g.map1 + no : g.map0 + no;
  int* map_out = (j & 1) ? g.map0 + no : g.map1 + no;
  for (int q = tid; q < n; q += BI_NT) mp[q] = __ldcg(map_in + q);
  __syncthreads();
  if (warp == 0) {
    double best = -1.0;
    int bi = n;
    const double* nrm_in = g.nrm + (j & 1) * g.ntot;
    for (int q = j + lane; q < n; q += 32) {
      double v = __ldcg(nrm_in + no + mp[q]);
      if (v > best) { best = v; bi = q; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) {
      double rjj = sqrt(best);
      double r00 = j == 0 ? rjj : __ldcg(g.r00 + b);
      int stop = j == 0 ? !(rjj > 0.0) : (rjj <= a.eps * r00);
      s_p = bi;
      s_rjj = rjj;
      s_r00 = r00;
      s_stop = stop;
    }
  }
  __syncthreads();
  const int64_t boff = a.off[b];
  if (s_stop) {
    if (cb == 0 && tid == 0) {
      g.kk[b] = j;
      for (int q = 0; q < n; ++q) lperm[boff + q] = mp[q];
    }
    return;
  }
  const int p = s_p;
  const double rjj = s_rjj;
  if (cb == 0 && tid == 0 && j == 0) g.r00[b] = s_r00;
  // exchange positions j and p
  if (tid == 0) {
    int t = mp[j];
    mp[j] = mp[p];
    mp[p] = t;
  }
  __syncthreads();
  if (cb == 0) {
    for (int q = tid; q < n; q += BI_NT) map_out[q] = mp[q];
    if (tid == 0 && j + 1 == kmax) {   // ran to the full rank: emit the order now
      for (int q = 0; q < n; ++q) lperm[boff + q] = mp[q];
    }
  }
  // reflector from the pivot column (rows j..m-1)
  const int pj = mp[j];
  const S* pcol = Mws + g.moff[b] + (size_t)pj * m;
  const S alpha = ldcg_s(pcol + j);
  const double aa = sqrt(abs2(alpha));
  const S phase = aa > 0.0 ? scal(alpha, 1.0 / aa) : S(1.0);
  const S beta = scal(phase, -rjj);
  for (int r = j + tid; r < m; r += BI_NT) u[r - j] = r == j ? alpha - beta : ldcg_s(pcol + r);
  const double f = 1.0 / (rjj * (rjj + aa));
  __syncthreads();
  // columns owned by this CTA that are still unpivoted (position > j)
  __shared__ int posof[CB];
  for (int cl = tid; cl < CB; cl += BI_NT) posof[cl] = -1;
  __syncthreads();
  for (int q = j + tid; q < n; q += BI_NT) {
    int c = mp[q];
    if (c >= cb * CB && c < cb * CB + CB) posof[c - cb * CB] = q;
  }
  __syncthreads();
  for (int cl = warp; cl < CB; cl += BI_NT / 32) {
    const int c = cb * CB + cl;
    const int q = posof[cl];
    if (c >= n || q < 0) continue;
    S* col = Mws + g.moff[b] + (size_t)c * m;
    S* cs = Ms ? Ms + (size_t)cl * m : col;
    if (q == j) {   // the pivot column: R_jj goes to rdiag (its rows are read by every CTA this step)
      if (lane == 0) reinterpret_cast<S*>(g.rdiag)[no + j] = beta;
      continue;
    }
    S s = S(0.0);
    for (int r = j + lane; r < m; r += 32) s += conj_(u[r - j]) * cs[r];
    s = warp_sum(s);
    s = shfl(s, 0);
    const S fs = scal(s, f);
    double s2 = 0.0;
    for (int r = j + lane; r < m; r += 32) {
      const S v = cs[r] - u[r - j] * fs;
      cs[r] = v;
      if (Ms) col[r] = v;
      if (r > j) s2 += abs2(v);
    }
    s2 = warp_sum(s2);
    if (lane == 0) g.nrm[((j + 1) & 1) * g.ntot + no + c] = s2;   // read by the next step only
  }
}

template <class S>
__global__ void __launch_bounds__(BI_NT) k_bbid_step(IdArgs a, BigId g, S* Mws, int j, int ncb, int* lperm) {
  bbid_body<S, BI_CB>(a, g, Mws, j, ncb, lperm, nullptr);
}

// All pivot steps of a level in one cooperative launch: a grid barrier
// between steps, and an exit once every box has found its rank.
template <class S, int CB>
__global__ void __launch_bounds__(BI_NT) k_bbid_coop(IdArgs a, BigId g, S* Mws, int nsteps, int ncb, int nb,
                                                     int* lperm, GridBar gb) {
  __shared__ int s_any;
  extern __shared__ __align__(16) unsigned char bi_smem[];
  // after u[mmax] | mp[nmax]: the CTA's own columns [CB][m]
  const size_t head = ((sizeof(S) * (size_t)a.mmax + sizeof(int) * (size_t)a.nmax) + 15) & ~(size_t)15;
  S* Ms = reinterpret_cast<S*>(bi_smem + head);
  {
    const int b = blockIdx.x / ncb, cb = blockIdx.x % ncb;
    const int n = a.n[b], m = g.m[b];
    const int nc = max(0, min(n, cb * CB + CB) - cb * CB);
    const S* src = Mws + g.moff[b] + (size_t)cb * CB * m;
    for (int e = threadIdx.x; e < nc * m; e += BI_NT) Ms[e] = src[e];
    __syncthreads();
  }
  for (int j = 0; j < nsteps; ++j) {
    bbid_body<S, CB>(a, g, Mws, j, ncb, lperm, Ms);
    if (!grid_sync(gb, (unsigned int)(j + 1) * gridDim.x)) return;
    if (threadIdx.x == 0) {
      int any = 0;
      for (int b = 0; b < nb && !any; ++b) {
        const int kmax = min(g.m[b], a.n[b]);
        if (__ldcg(g.kk + b) == kmax && j + 1 < kmax) any = 1;
      }
      s_any = any;
    }
    __syncthreads();
    if (!s_any) return;
  }
}

// The pivoted QR of every box of a level on a thread-block cluster of CTAs
// (one cluster per box).  CTA q keeps the box's physical columns
// [q cw, q cw + cw) in shared memory for the whole factorization.  Each step:
// every CTA publishes its best trailing column (exact norm, lowest position on
// ties) with that column's row-j entry; after one cluster barrier all CTAs
// read the candidates through distributed shared memory, agree on the pivot
// and form the same reflector coefficients, copy the pivot column from its
// owner (which does not change it this step), apply the reflector to their
// own columns and recompute their trailing norms.  One cluster barrier per
// step and no grid-wide barrier.  Output as the cooperative kernel: rows 0..k-1 of the columns in
// Mws, R_jj in rdiag, the rank in kk, the column order in lperm.
template <class S>
__global__ void __launch_bounds__(BI_NT) k_bbid_cluster(IdArgs a, BigId g, S* Mws, int cw, int* lperm) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char bc_smem[];
  __shared__ double s_r00, s_f;
  __shared__ S s_u0;
  __shared__ int s_p, s_stop, s_owner;
  const int cs = (int)cl.num_blocks(), q = (int)cl.block_rank();
  const int b = blockIdx.x / cs;
  const int n = a.n[b], m = g.m[b];
  const int kmax = min(m, n);
  const int c_beg = q * cw, nc = max(0, min(n, c_beg + cw) - c_beg);
  // Ms[cw][m] | u[mmax] | canda[2] | nrm[cw] | candv[2] | pos[nmax] | posof[cw] | candp[2]
  S* Ms = reinterpret_cast<S*>(bc_smem);
  S* u = Ms + (size_t)cw * a.mmax;
  S* canda = u + a.mmax;
  double* nrm = reinterpret_cast<double*>(canda + 2);
  double* candv = nrm + cw;
  int* pos = reinterpret_cast<int*>(candv + 2);
  int* posof = pos + a.nmax;
  int* candp = posof + cw;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = BI_NT / 32, QG = 8, QCW = 32 / QG;
  const int gl = lane & (QG - 1), grp = lane / QG;
  const S* src = Mws + g.moff[b] + (size_t)c_beg * m;
  for (int e = tid; e < nc * m; e += BI_NT) Ms[e] = src[e];
  for (int i = tid; i < n; i += BI_NT) pos[i] = i;
  for (int i = tid; i < nc; i += BI_NT) posof[i] = c_beg + i;
  __syncthreads();
  for (int cb = warp * QCW; cb < nc; cb += NW * QCW) {   // exact column norms
    const int c = cb + grp;
    const bool act = c < nc;
    double s2 = 0.0;
    if (act)
      for (int r = gl; r < m; r += QG) s2 += abs2(Ms[(size_t)c * m + r]);
    s2 = group_sum<QG>(s2);
    if (act && gl == 0) nrm[c] = s2;
  }
  __syncthreads();
  auto better = [](double v, int p, double bv, int bp) { return v > bv || (v == bv && p < bp); };
  int j = 0;
  for (; j < kmax; ++j) {
    if (warp == 0) {   // this CTA's candidate
      double best = -1.0;
      int bp = n, bi = 0;
      for (int i = lane; i < nc; i += 32) {
        const int ps = posof[i];
        if (ps >= j && better(nrm[i], ps, best, bp)) { best = nrm[i]; bp = ps; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, bp, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (better(ob, op, best, bp)) { best = ob; bp = op; bi = oi; }
      }
      if (lane == 0) {
        candv[j & 1] = best;
        candp[j & 1] = bp;
        canda[j & 1] = nc > 0 ? Ms[(size_t)bi * m + j] : S(0.0);
      }
    }
    cl.sync();
    if (warp == 0) {   // the cluster's pivot and reflector (the same in every CTA)
      double best = -1.0;
      int bp = n, br = 0;
      if (lane < cs) {
        best = cl.map_shared_rank(candv, lane)[j & 1];
        bp = cl.map_shared_rank(candp, lane)[j & 1];
        br = lane;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, bp, o);
        const int orr = __shfl_xor_sync(0xffffffffu, br, o);
        if (better(ob, op, best, bp)) { best = ob; bp = op; br = orr; }
      }
      if (lane == 0) {
        const double rjj = sqrt(fmax(best, 0.0));
        const double r00 = j == 0 ? rjj : s_r00;
        const int stop = j == 0 ? !(rjj > 0.0) : (rjj <= a.eps * r00);
        s_r00 = r00;
        s_stop = stop;
        if (!stop) {
          // Householder reflector H = I - f u u^H of the pivot column (rows
          // j..m-1): beta = -phase(alpha) rjj, u = x - beta e_1
          const S alpha = cl.map_shared_rank(canda, br)[j & 1];
          const double aa = sqrt(abs2(alpha));
          const S phase = aa > 0.0 ? scal(alpha, 1.0 / aa) : S(1.0);
          const S beta = scal(phase, -rjj);
          s_u0 = alpha - beta;
          s_f = 1.0 / (rjj * (rjj + aa));
          const int pc = pos[bp], cj = pos[j];   // exchange positions j and bp
          pos[j] = pc;
          pos[bp] = cj;
          if (cj >= c_beg && cj < c_beg + nc) posof[cj - c_beg] = bp;
          if (pc >= c_beg && pc < c_beg + nc) posof[pc - c_beg] = j;
          s_p = pc;
          s_owner = pc / cw;
          if (q == pc / cw) reinterpret_cast<S*>(g.rdiag)[g.noff[b] + j] = beta;
        }
      }
    }
    __syncthreads();
    if (s_stop) break;   // uniform over the cluster
    const int pc = s_p, owner = s_owner;
    {   // u from the pivot column, which its owner leaves unchanged this step
      const S* pcol = cl.map_shared_rank(Ms + (size_t)(pc - owner * cw) * m, owner);
      for (int r = j + 1 + tid; r < m; r += BI_NT) u[r - j] = pcol[r];
      if (tid == 0) u[0] = s_u0;
    }
    __syncthreads();
    const double f = s_f;
    for (int cb = warp * QCW; cb < nc; cb += NW * QCW) {   // own unpivoted columns
      const int c = cb + grp;
      const bool act = c < nc && posof[c] > j;
      S* col = Ms + (size_t)(act ? c : 0) * m;
      S sd = S(0.0);
      if (act)
        for (int r = j + gl; r < m; r += QG) sd += conj_(u[r - j]) * col[r];
      sd = group_sum<QG>(sd);
      const S fs = scal(sd, f);
      double s2 = 0.0;
      if (act)
        for (int r = j + gl; r < m; r += QG) {
          const S v = col[r] - u[r - j] * fs;
          col[r] = v;
          if (r > j) s2 += abs2(v);
        }
      s2 = group_sum<QG>(s2);
      if (act && gl == 0) nrm[c] = s2;
    }
    __syncthreads();
  }
  const int k = j;
  S* dst = Mws + g.moff[b] + (size_t)c_beg * m;
  for (int e = tid; e < nc * k; e += BI_NT) {
    const int c = e / k, r = e % k;
    dst[(size_t)c * m + r] = Ms[(size_t)c * m + r];
  }
  if (q == 0) {
    for (int i = tid; i < n; i += BI_NT) lperm[a.off[b] + i] = pos[i];
    if (tid == 0) {
      g.kk[b] = k;
      g.r00[b] = s_r00;
    }
  }
  cl.sync();   // no CTA leaves while another may still read its shared memory
}

// 1 if some box of the level is still pivoting at step j.
__global__ void k_bbid_active(BigId g, const int* n, int nb, int j, int* out) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    int kmax = min(g.m[b], n[b]);
    if (g.kk[b] == kmax && j < kmax) any = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) *out = any;
}

// T = R11^-1 R12 for every column of R12 (one warp per column), ranks out.
template <class S>
__global__ void k_bbid_T(IdArgs a, BigId g, const S* Mws, S* Tpool, int tiles_per_box) {
  const int b = blockIdx.x / tiles_per_box;
  const int e = (blockIdx.x % tiles_per_box) * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int n = a.n[b], m = g.m[b], k = g.kk[b];
  if (blockIdx.x % tiles_per_box == 0 && threadIdx.x == 0) a.kout[b] = k;
  if (e >= n - k) return;
  const int* lp = a.lperm + a.off[b];
  const S* M = Mws + g.moff[b];
  S* T = Tpool + a.toff[b];
  const S* rhs = M + (size_t)lp[k + e] * m;
  // t = R11^-1 rhs[0:k] with R11[i][i'] = M[i, lp[i']] (column-oriented, lane-parallel updates)
  S* t = T + (size_t)e * k;
  for (int i = lane; i < k; i += 32) t[i] = rhs[i];
  __syncwarp();
  for (int i = k - 1; i >= 0; --i) {
    const S* ci = M + (size_t)lp[i] * m;
    S ti = S(0.0);
    if (lane == 0) {
      ti = t[i] / reinterpret_cast<const S*>(g.rdiag)[g.noff[b] + i];
      t[i] = ti;
    }
    ti = shfl(ti, 0);
    __syncwarp();
    for (int r = lane; r < i; r += 32) t[r] -= ci[r] * ti;
    __syncwarp();
  }
}

// Gauss-Jordan with partial pivoting on the augmented n x 2n matrix [A | I]
// (column-major, ld = n); leaves A^-1 in the right half.  Sets *bad on a zero
// or non-finite pivot.
template <class S, int NT>
__device__ void gauss_jordan(S* A, int n, S* mult, int* bad) {
  __shared__ int s_p;
  __shared__ double s_best;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ld = n, w = 2 * n;
  for (int j = 0; j < n; ++j) {
    if (warp == 0) {
      double best = -1.0;
      int bi = j;
      for (int r = j + lane; r < n; r += 32) {
        double v = abs2(A[r + (size_t)j * ld]);
        if (v > best) { best = v; bi = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) { s_p = bi; s_best = best; }
    }
    __syncthreads();
    const int p = s_p;
    if (!(s_best > 0.0) || !isfinite(s_best)) {
      if (tid == 0) atomicOr(bad, 1);
      __syncthreads();
      continue;
    }
    if (p != j)
      for (int c = tid; c < w; c += NT) {
        S t = A[j + (size_t)c * ld];
        A[j + (size_t)c * ld] = A[p + (size_t)c * ld];
        A[p + (size_t)c * ld] = t;
      }
    __syncthreads();
    const S inv = S(1.0) / A[j + (size_t)j * ld];
    __syncthreads();
    for (int c = j + tid; c < w; c += NT) A[j + (size_t)c * ld] = A[j + (size_t)c * ld] * inv;
    for (int r = tid; r < n; r += NT) mult[r] = A[r + (size_t)j * ld];
    __syncthreads();
    const int64_t cnt = (int64_t)(w - j - 1) * n;
    for (int64_t e = tid; e < cnt; e += NT) {
      int r = (int)(e % n);
      int c = j + 1 + (int)(e / n);
      if (r != j) A[r + (size_t)c * ld] -= mult[r] * A[j + (size_t)c * ld];
    }
    __syncthreads();
  }
}

struct FaArgs {
  KParams kp;
  Pts pts;
  int leaf_level;         // 1: D = A(I, I)
  const int* n;
  const int* k;
  const int64_t* off;
  const int* act;
  const int* owner;       // child box of each active position (upper levels)
  const int64_t* cskoff;  // children's skeleton offsets (depth + 1)
  const int* ck;          // children's ranks
  const int64_t* clamoff; // children's Lambda offsets
  const int* lperm;
  const int64_t* toff;
  const int64_t* wsoff;
  const int64_t* uoff;
  const int64_t* loff;
  const int64_t* lamoff;
  int* bad;
  // forward-operator rows [D ; P]: real kernels float (fu32) and double-float
  // (fudf); complex kernels complex float and complex double-float in the
  // same slots
  float* fu32;
  dfloat* fudf;
  // non-symmetric kernels (general = 1, k_factor only): rows of D from the
  // row active set, L = Q^T from the row ID (lperm_r, Tr at toff)
  int general;
  const int* act_r;
  const int* lperm_r;
  const void* Tr;
};

// The forward operator's D block shares the assembled block's entries: the
// same at the leaves; above, zero inside one child's block (where the
// assembled block holds the child's Lambda).  Written while assembling into
// rows 0..n-1 of FU ((n+k) x n at uoff): float and double-float for real
// kernels, complex float and complex double-float for complex ones.
template <class S>
__device__ __forceinline__ void emit_fwd(const FaArgs& a, int b, int n, int k, int r, int c, S v, bool same_child) {
  if (!a.fu32) return;
  const int64_t i = a.uoff[b] + r + (int64_t)c * (n + k);
  if constexpr (std::is_same<S, double>::value) {
    const double f = (a.leaf_level || !same_child) ? v : 0.0;
    a.fu32[i] = f64_to_f32_rn(f);
    a.fudf[i] = f64_to_df(f);
  } else {
    const S f = (a.leaf_level || !same_child) ? v : S(0.0);
    reinterpret_cast<c64*>(a.fu32)[i] = c64(f64_to_f32_rn(f.re), f64_to_f32_rn(f.im));
    reinterpret_cast<cdfloat*>(a.fudf)[i] = cdfloat(f64_to_df(f.re), f64_to_df(f.im));
  }
}

template <class S, int NT>
__global__ void __launch_bounds__(NT) k_factor(FaArgs a, const S* Tpool, const S* cLam, S* ws, S* Upool,
                                               S* Lpool, S* Lampool) {
  extern __shared__ __align__(16) unsigned char smem[];
  S* mult = reinterpret_cast<S*>(smem);
  const int b = blockIdx.x, tid = threadIdx.x;
  const int n = a.n[b], k = a.k[b], nr = n - k;
  const int64_t off = a.off[b];
  const int* lp = a.lperm + off;
  const S* T = Tpool + (a.toff ? a.toff[b] : 0);
  S* Aug = ws + a.wsoff[b];
  S* X = Aug + (size_t)2 * n * n;
  S* Y = X + (size_t)n * k;
  S* Yr = Y + (size_t)2 * k * k;   // general: P D^-1 (k x n)
  const int* lpr = a.general ? a.lperm_r + off : lp;
  const S* Tq = a.general ? reinterpret_cast<const S*>(a.Tr) + (a.toff ? a.toff[b] : 0) : T;
  const int* act_rows = a.general ? a.act_r : a.act;

  // D (left half) and I (right half)
  for (int64_t e = tid; e < (int64_t)n * n; e += NT) {
    int r = (int)(e % n), c = (int)(e / n);
    int pr = act_rows[off + r], pc = a.act[off + c];
    S v;
    if (a.leaf_level) {
      v = system_entry<S>(a.kp, a.pts, pr, pc);
    } else {
      int orow = a.owner[off + r], ocol = a.owner[off + c];
      if (orow == ocol) {
        int64_t base = a.cskoff[orow];
        int kc = a.ck[orow];
        v = cLam[a.clamoff[orow] + (off + r - base) + (int64_t)(off + c - base) * kc];
      } else {
        v = offdiag_entry<S>(a.kp, a.pts, pr, pc);
      }
    }
    Aug[r + (size_t)c * n] = v;
    Aug[r + (size_t)(n + c) * n] = (r == c) ? S(1.0) : S(0.0);
    emit_fwd<S>(a, b, n, k, r, c, v, !a.leaf_level && a.owner[off + r] == a.owner[off + c]);
  }
  __syncthreads();
  gauss_jordan<S, NT>(Aug, n, mult, a.bad);
  const S* Dinv = Aug + (size_t)n * n;
  S* U = Upool + a.uoff[b];        // (n + k) x n, ld n + k
  const int ldu = n + k;
  if (k == 0) {
    for (int64_t e = tid; e < (int64_t)n * n; e += NT) {
      int r = (int)(e % n), c = (int)(e / n);
      U[r + (size_t)c * ldu] = Dinv[r + (size_t)c * n];
    }
    return;
  }
  // X = D^-1 L = D^-1 Q^T : X[:, i] = Dinv[:, sk_i] + sum_e T[i, e] Dinv[:, rd_e]
  // (the row ID's skeletons and T; Q = P for symmetric kernels)
  for (int64_t e = tid; e < (int64_t)n * k; e += NT) {
    int r = (int)(e % n), i = (int)(e / n);
    S s = Dinv[r + (size_t)lpr[i] * n];
    for (int q = 0; q < nr; ++q) s += Tq[i + (size_t)q * k] * Dinv[r + (size_t)lpr[k + q] * n];
    X[r + (size_t)i * n] = s;
  }
  if (a.general)   // Yr = R D^-1 = P D^-1 : Yr[i, c] = Dinv[sk_i, c] + sum_e T[i, e] Dinv[rd_e, c]
    for (int64_t e = tid; e < (int64_t)k * n; e += NT) {
      int i = (int)(e % k), c = (int)(e / k);
      S s = Dinv[lp[i] + (size_t)c * n];
      for (int q = 0; q < nr; ++q) s += T[i + (size_t)q * k] * Dinv[lp[k + q] + (size_t)c * n];
      Yr[i + (size_t)c * k] = s;
    }
  __syncthreads();
  // [P X | I] : (P X)[i, c] = X[sk_i, c] + sum_e T[i, e] X[rd_e, c]
  for (int64_t e = tid; e < (int64_t)k * k; e += NT) {
    int i = (int)(e % k), c = (int)(e / k);
    S s = X[lp[i] + (size_t)c * n];
    for (int q = 0; q < nr; ++q) s += T[i + (size_t)q * k] * X[lp[k + q] + (size_t)c * n];
    Y[i + (size_t)c * k] = s;
    Y[i + (size_t)(k + c) * k] = (i == c) ? S(1.0) : S(0.0);
  }
  __syncthreads();
  gauss_jordan<S, NT>(Y, k, mult, a.bad);
  const S* Lam = Y + (size_t)k * k;
  S* Lo = Lampool + a.lamoff[b];
  for (int e = tid; e < k * k; e += NT) Lo[e] = Lam[e];
  // calL = X Lambda  (n x k)
  S* Lf = Lpool + a.loff[b];
  for (int64_t e = tid; e < (int64_t)n * k; e += NT) {
    int r = (int)(e % n), c = (int)(e / n);
    S s = S(0.0);
    for (int q = 0; q < k; ++q) s += X[r + (size_t)q * n] * Lam[q + (size_t)c * k];
    Lf[r + (size_t)c * n] = s;
  }
  // calR = Lambda R D^-1 (k x n) -> rows n.. of U: R D^-1 = X^T for a
  // symmetric D and Q = P, else Yr
  for (int64_t e = tid; e < (int64_t)k * n; e += NT) {
    int i = (int)(e % k), c = (int)(e / k);
    S s = S(0.0);
    if (a.general)
      for (int q = 0; q < k; ++q) s += Lam[i + (size_t)q * k] * Yr[q + (size_t)c * k];
    else
      for (int q = 0; q < k; ++q) s += Lam[i + (size_t)q * k] * X[c + (size_t)q * n];
    U[n + i + (size_t)c * ldu] = s;
  }
  __syncthreads();
  // calD = Dinv - calL R D^-1  (n x n) -> rows 0..n-1 of U
  for (int64_t e = tid; e < (int64_t)n * n; e += NT) {
    int r = (int)(e % n), c = (int)(e / n);
    S s = Dinv[r + (size_t)c * n];
    if (a.general)
      for (int q = 0; q < k; ++q) s -= Lf[r + (size_t)q * n] * Yr[q + (size_t)c * k];
    else
      for (int q = 0; q < k; ++q) s -= Lf[r + (size_t)q * n] * X[c + (size_t)q * n];
    U[r + (size_t)c * ldu] = s;
  }
}

// In-place Gauss-Jordan inversion with partial pivoting of the n x n
// column-major matrix A (shared memory): n^3 multiply-adds.  Rows are
// swapped as pivots are chosen and the columns unscrambled at the end.
template <class S, int NT>
__device__ void gj_inplace(S* A, int n, S* mult, int* piv, int* bad) {
  __shared__ int s_p;
  __shared__ double s_best;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = 0; j < n; ++j) {
    if (warp == 0) {
      double best = -1.0;
      int bi = j;
      for (int r = j + lane; r < n; r += 32) {
        double v = abs2(A[r + j * n]);
        if (v > best) { best = v; bi = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) { s_p = bi; s_best = best; piv[j] = bi; }
    }
    __syncthreads();
    if (!(s_best > 0.0) || !isfinite(s_best)) {
      if (tid == 0) atomicOr(bad, 1);
      __syncthreads();
      continue;
    }
    const int p = s_p;
    if (p != j)
      for (int c = tid; c < n; c += NT) {
        S t = A[j + c * n];
        A[j + c * n] = A[p + c * n];
        A[p + c * n] = t;
      }
    __syncthreads();
    const S inv = S(1.0) / A[j + j * n];
    for (int r = tid; r < n; r += NT) {
      mult[r] = A[r + j * n];
      A[r + j * n] = r == j ? S(1.0) : S(0.0);
    }
    __syncthreads();
    for (int c = tid; c < n; c += NT) A[j + c * n] = A[j + c * n] * inv;
    __syncthreads();
    for (int e = tid; e < n * n; e += NT) {
      int r = e % n, c = e / n;
      if (r != j) A[r + c * n] -= mult[r] * A[j + c * n];
    }
    __syncthreads();
  }
  for (int j = n - 1; j >= 0; --j) {
    const int p = piv[j];
    if (p != j)
      for (int r = tid; r < n; r += NT) {
        S t = A[r + j * n];
        A[r + j * n] = A[r + p * n];
        A[r + p * n] = t;
      }
    __syncthreads();
  }
}

// Entry e of the upper triangle of an n x n matrix, column by column:
// (r, c) with r <= c, e = c (c + 1) / 2 + r.
__device__ __forceinline__ void tri_index(int e, int& r, int& c) {
  int cc = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while ((cc + 1) * (cc + 2) / 2 <= e) ++cc;
  while (cc * (cc + 1) / 2 > e) --cc;
  c = cc;
  r = e - cc * (cc + 1) / 2;
}

// The block elimination of k_factor with every intermediate in shared
// memory: [D^-1 (n x n) | X (n x k) | (PX)^-1 (k x k) | mult (n) | piv (n)].
template <class S, int NT>
__global__ void __launch_bounds__(NT) k_factor_smem(FaArgs a, const S* Tpool, const S* cLam, S* Upool, S* Lpool,
                                                    S* Lampool) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int b = blockIdx.x, tid = threadIdx.x;
  const int n = a.n[b], k = a.k[b], nr = n - k;
  const int64_t off = a.off[b];
  const int* lp = a.lperm + off;
  const S* T = Tpool + (a.toff ? a.toff[b] : 0);
  S* Dv = reinterpret_cast<S*>(smem);
  S* X = Dv + (size_t)n * n;
  S* Y = X + (size_t)n * k;
  S* mult = Y + (size_t)k * k;
  int* piv = reinterpret_cast<int*>(mult + n);

  // D is symmetric (the kernels are, and so are the children's Lambda blocks
  // up to rounding): one triangle, mirrored
  for (int e = tid; e < n * (n + 1) / 2; e += NT) {
    int r, c;
    tri_index(e, r, c);
    int pr = a.act[off + r], pc = a.act[off + c];
    S v;
    if (a.leaf_level) {
      v = system_entry<S>(a.kp, a.pts, pr, pc);
    } else {
      int orow = a.owner[off + r], ocol = a.owner[off + c];
      if (orow == ocol) {
        int64_t base = a.cskoff[orow];
        int kc = a.ck[orow];
        v = cLam[a.clamoff[orow] + (off + r - base) + (int64_t)(off + c - base) * kc];
      } else {
        v = offdiag_entry<S>(a.kp, a.pts, pr, pc);
      }
    }
    const bool same = !a.leaf_level && a.owner[off + r] == a.owner[off + c];
    Dv[r + c * n] = v;
    emit_fwd<S>(a, b, n, k, r, c, v, same);
    if (r != c) {
      Dv[c + r * n] = v;
      emit_fwd<S>(a, b, n, k, c, r, v, same);
    }
  }
  __syncthreads();
  gj_inplace<S, NT>(Dv, n, mult, piv, a.bad);    // Dv = D^-1
  S* U = Upool + a.uoff[b];
  const int ldu = n + k;
  if (k == 0) {
    for (int e = tid; e < n * n; e += NT) U[(e % n) + (size_t)(e / n) * ldu] = Dv[e];
    return;
  }
  // X = D^-1 P^T
  for (int e = tid; e < n * k; e += NT) {
    int r = e % n, i = e / n;
    S s = Dv[r + lp[i] * n];
    for (int q = 0; q < nr; ++q) s += T[i + (size_t)q * k] * Dv[r + lp[k + q] * n];
    X[e] = s;
  }
  __syncthreads();
  // Y = P X = P D^-1 P^T (symmetric: one triangle, mirrored), then
  // Lambda = Y^-1 in place
  for (int e = tid; e < k * (k + 1) / 2; e += NT) {
    int i, c;
    tri_index(e, i, c);
    S s = X[lp[i] + c * n];
    for (int q = 0; q < nr; ++q) s += T[i + (size_t)q * k] * X[lp[k + q] + c * n];
    Y[i + c * k] = s;
    Y[c + i * k] = s;
  }
  __syncthreads();
  gj_inplace<S, NT>(Y, k, mult, piv, a.bad);
  S* Lo = Lampool + a.lamoff[b];
  for (int e = tid; e < k * k; e += NT) Lo[e] = Y[e];
  // calL = X Lambda -> global; calR = Lambda X^T = calL^T (Lambda is
  // symmetric) -> rows n.. of U
  S* Lf = Lpool + a.loff[b];
  for (int e = tid; e < n * k; e += NT) {
    int r = e % n, c = e / n;
    S s = S(0.0);
    for (int q = 0; q < k; ++q) s += X[r + q * n] * Y[q + c * k];
    Lf[e] = s;
    U[n + c + (size_t)r * ldu] = s;
  }
  // calD = D^-1 - calL X^T = D^-1 - X Lambda X^T (symmetric: one triangle,
  // mirrored), reading back the calL just written
  __syncthreads();
  for (int e = tid; e < n * (n + 1) / 2; e += NT) {
    int r, c;
    tri_index(e, r, c);
    S s = Dv[r + c * n];
    for (int q = 0; q < k; ++q) s -= Lf[r + (size_t)q * n] * X[c + q * n];
    U[r + (size_t)c * ldu] = s;
    U[c + (size_t)r * ldu] = s;
  }
}

// ---------------------------------------------------------- big boxes
// Boxes too large for one CTA's shared memory (the top levels) are
// factored by many CTAs: the Gauss-Jordan inversion runs one launch per pivot
// step with each CTA owning 32 columns of one box, and the products of the
// block elimination run column-parallel.  Workspace per box (offset bo[b]):
// A (n x n, inverted in place) | Dinv (n x n) | X (n x k) | Y (k x k) |
// pivot column buffers (2 n) | pivots (n, stored as scalars' worth of ints).
struct BigArgs {
  int n_box;
  const int* n;
  const int* k;
  const int64_t* bo;       // workspace offset of each box (scalars)
};

constexpr int BB_NT = 128;
constexpr int BB_CB = 8;   // columns per CTA in a pivot step
constexpr int UNS_CB = 16; // columns per CTA of the final column permutation
constexpr int GJB_NT = 256;          // threads of the blocked Gauss-Jordan kernels
constexpr int GJB_APPLY_MAXC = 32;   // columns per CTA of k_gjb_apply, at most (shared memory permitting)

template <class S>
__device__ inline S* bb_A(S* ws, const BigArgs& g, int b) { return ws + g.bo[b]; }

// D of every box into A, column 0 into the first pivot buffer.
template <class S>
__global__ void k_bb_assemble(FaArgs a, BigArgs g, const S* cLam, S* ws, int maxn) {
  const int b = blockIdx.x / maxn, c = blockIdx.x % maxn;
  const int n = g.n[b];
  if (c >= n) return;
  const int k = g.k[b];
  const int64_t off = a.off[b];
  S* A = bb_A(ws, g, b);
  S* buf = A + 2 * (size_t)n * n + (size_t)n * k + (size_t)k * k;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    int pr = a.act[off + r], pc = a.act[off + c];
    S v;
    if (a.leaf_level) {
      v = system_entry<S>(a.kp, a.pts, pr, pc);
    } else {
      int orow = a.owner[off + r], ocol = a.owner[off + c];
      if (orow == ocol) {
        int64_t base = a.cskoff[orow];
        int kc = a.ck[orow];
        v = cLam[a.clamoff[orow] + (off + r - base) + (int64_t)(off + c - base) * kc];
      } else {
        v = offdiag_entry<S>(a.kp, a.pts, pr, pc);
      }
    }
    A[r + (size_t)c * n] = v;
    if (c == 0) buf[r] = v;
    emit_fwd<S>(a, b, n, k, r, c, v, !a.leaf_level && a.owner[off + r] == a.owner[off + c]);
  }
}

// One Gauss-Jordan step j on matrices M (m x m, ld m) of every box:
// M = base(b) + moff, size m = mdim(b).  The pivot column (before the step)
// is read from pbuf[j % 2]; the owner of column j+1 writes it, updated, to
// pbuf[(j+1) % 2].  Every CTA finds the same pivot.
template <class S, class Dims>
__device__ void bb_gj_body(const BigArgs& g, S* ws, const Dims& dims, int j, int ncb, int* bad) {
  extern __shared__ __align__(16) unsigned char bb_smem[];
  S* mult = reinterpret_cast<S*>(bb_smem);   // m entries
  __shared__ int s_p;
  __shared__ double s_best;
  const int b = blockIdx.x / ncb, cb = blockIdx.x % ncb;
  int m;
  S *M, *pb_in, *pb_out;
  int* piv;
  dims(ws, g, b, j, m, M, pb_in, pb_out, piv);
  if (j >= m || cb * BB_CB >= m) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (warp == 0) {
    double best = -1.0;
    int bi = j;
    for (int r = j + lane; r < m; r += 32) {
      double v = abs2(ldcg_s(pb_in + r));
      if (v > best) { best = v; bi = r; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { s_p = bi; s_best = best; }
  }
  __syncthreads();
  if (!(s_best > 0.0) || !isfinite(s_best)) {
    if (tid == 0 && cb == 0) atomicOr(bad, 1);
    return;
  }
  const int p = s_p;
  if (tid == 0 && cb == 0) piv[j] = p;
  for (int r = tid; r < m; r += BB_NT) mult[r] = ldcg_s(pb_in + (r == j ? p : (r == p ? j : r)));
  __syncthreads();
  const S inv = S(1.0) / mult[j];
  const int c_beg = cb * BB_CB, c_end = min(m, c_beg + BB_CB), nc = c_end - c_beg;
  __shared__ S newj[BB_CB];
  for (int cl = tid; cl < nc; cl += BB_NT) {
    const int c = c_beg + cl;
    newj[cl] = c == j ? inv : M[p + (size_t)c * m] * inv;   // row p moves to row j
  }
  __syncthreads();
  // rows other than j keep their position, row p receives old row j; the
  // pivot column itself is e_j transformed (identity trick of in-place GJ)
  for (int e = tid; e < nc * m; e += BB_NT) {
    const int r = e % m, cl = e / m, c = c_beg + cl;
    if (r == j) continue;
    S* col = M + (size_t)c * m;
    const S old = c == j ? S(0.0) : (r == p ? col[j] : col[r]);
    const S v = old - mult[r] * newj[cl];
    col[r] = v;
    if (c == j + 1) pb_out[r] = v;
  }
  __syncthreads();
  for (int cl = tid; cl < nc; cl += BB_NT) {
    const int c = c_beg + cl;
    M[j + (size_t)c * m] = newj[cl];
    if (c == j + 1) pb_out[j] = newj[cl];
  }
}

// Blocked form of the same in-place Gauss-Jordan for one large box (the
// root): the m steps in panels of GJB columns.  k_gjb_panel runs a panel's
// steps on the panel columns alone (one CTA).  For any other column a, the
// panel's steps amount to a -> Pi a + V (Pi a)[panel rows], with Pi the
// panel's row exchanges in order and V = (panel after its steps) - (identity
// columns of the panel rows) -- the in-place panel holds the panel's
// transformation applied to the unit vectors it replaced.  k_gjb_apply does
// that rank-GJB update for all other columns at once.  Two launches per panel
// instead of a barrier per step.
constexpr int GJB = 16;

// Magnitude key of a pivot candidate: |x| as ordered bits for real entries
// (integer compares), |x|^2 for complex ones.
__device__ inline double piv_key(double x) { return fabs(x); }
__device__ inline double piv_key(c128 x) { return abs2(x); }

template <class S, class Dims>
__global__ void __launch_bounds__(GJB_NT) k_gjb_panel(BigArgs g, S* ws, Dims dims, int c0, int in_smem, int* bad) {
  extern __shared__ __align__(16) unsigned char gp_smem[];
  __shared__ int s_p, s_fail;
  __shared__ S s_inv;
  __shared__ S newj[GJB], rowj[GJB];
  int m;
  S *M, *pb_in, *pb_out;
  int* piv;
  dims(ws, g, blockIdx.x, 0, m, M, pb_in, pb_out, piv);   // one CTA per box
  if (c0 >= m) return;
  const int bw = min(GJB, m - c0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  S* mult = reinterpret_cast<S*>(gp_smem);                  // m entries
  S* P = in_smem ? mult + m : M + (size_t)c0 * m;           // the panel, ld m
  if (in_smem)
    for (int e = tid; e < bw * m; e += GJB_NT) P[e] = M[(size_t)c0 * m + e];
  if (tid == 0) s_fail = 0;
  __syncthreads();
  for (int jj = 0; jj < bw; ++jj) {
    const int j = c0 + jj;
    const S* colj = P + (size_t)jj * m;
    if (warp == 0) {   // pivot: largest magnitude in rows j..m-1, lowest row on ties
      long long best = -1;
      int bi = j;
      for (int r = j + lane; r < m; r += 32) {
        const long long v = __double_as_longlong(piv_key(colj[r]));
        if (v > best) { best = v; bi = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        const double bv = __longlong_as_double(best);
        s_p = bi;
        if (!(bv > 0.0) || !isfinite(bv)) s_fail = 1;
        else s_inv = S(1.0) / colj[bi];
      }
    }
    __syncthreads();
    if (s_fail) break;
    const int p = s_p;
    const S inv = s_inv;
    for (int r = tid; r < m; r += GJB_NT) mult[r] = colj[r == j ? p : (r == p ? j : r)];
    for (int cl = tid; cl < bw; cl += GJB_NT) {
      newj[cl] = cl == jj ? inv : P[p + (size_t)cl * m] * inv;
      rowj[cl] = P[j + (size_t)cl * m];
    }
    if (tid == 0) piv[j] = p;
    __syncthreads();
    for (int r = tid; r < m; r += GJB_NT) {
      const S mr = mult[r];
      for (int cl = 0; cl < bw; ++cl) {
        S* col = P + (size_t)cl * m;
        if (r == j) {
          col[j] = newj[cl];
          continue;
        }
        const S old = cl == jj ? S(0.0) : (r == p ? rowj[cl] : col[r]);
        col[r] = old - mr * newj[cl];
      }
    }
    __syncthreads();
  }
  if (s_fail) {
    if (tid == 0) atomicOr(bad, 1);
    return;
  }
  if (in_smem)
    for (int e = tid; e < bw * m; e += GJB_NT) M[(size_t)c0 * m + e] = P[e];
}

// The panel steps of k_gjb_panel on a thread-block cluster per box: CTA q
// keeps rows [q rpc, q rpc + rpc) of the panel in shared memory.  A step:
// every CTA publishes its largest candidate (magnitude bits, lowest row on
// ties) with a copy of that row, and the owner of row j a copy of row j
// (both double-buffered by step parity); after one cluster barrier all CTAs
// agree on the pivot row p, read the two copies from their owners and apply
// the step to their own rows.  The copies are never written while they may
// be read: a CTA writes the same parity again only two steps later, after
// the next barrier, by which time every CTA has read them.
template <class S, class Dims>
__global__ void __launch_bounds__(GJB_NT) k_gjb_panel_cl(BigArgs g, S* ws, Dims dims, int c0, int rpc, int* bad) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char gc_smem[];
  __shared__ long long s_key[GJB_NT / 32];
  __shared__ int s_row[GJB_NT / 32];
  __shared__ long long cand_k[2];
  __shared__ int cand_r[2];
  __shared__ int s_p, s_fail;
  __shared__ S rowp[GJB], rowj[GJB], newj[GJB];
  __shared__ S pub_p[2][GJB], pub_j[2][GJB];   // copies of the candidate row and of row j
  const int cs = (int)cl.num_blocks(), q = (int)cl.block_rank();
  int m;
  S *M, *pb_in, *pb_out;
  int* piv;
  dims(ws, g, blockIdx.x / cs, 0, m, M, pb_in, pb_out, piv);
  if (c0 >= m) return;   // uniform over the cluster (same box)
  const int bw = min(GJB, m - c0);
  const int r0 = q * rpc, nr = max(0, min(m, r0 + rpc) - r0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  S* P = reinterpret_cast<S*>(gc_smem);   // [bw][rpc]: column cl of the panel, local rows
  for (int e = tid; e < bw * nr; e += GJB_NT) {
    const int c = e / nr, rl = e % nr;
    P[(size_t)c * rpc + rl] = M[(r0 + rl) + (size_t)(c0 + c) * m];
  }
  if (tid == 0) s_fail = 0;
  __syncthreads();
  for (int jj = 0; jj < bw; ++jj) {
    const int j = c0 + jj;
    const S* colj = P + (size_t)jj * rpc;
    {   // this CTA's candidate among its rows >= j
      long long best = -1;
      int bi = m;
      for (int rl = tid; rl < nr; rl += GJB_NT) {
        if (r0 + rl < j) continue;
        const long long v = __double_as_longlong(piv_key(colj[rl]));
        if (v > best) { best = v; bi = r0 + rl; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) { s_key[warp] = best; s_row[warp] = bi; }
      __syncthreads();
      if (tid == 0) {
        long long bk = s_key[0];
        int br = s_row[0];
        for (int w = 1; w < GJB_NT / 32; ++w)
          if (s_key[w] > bk || (s_key[w] == bk && s_row[w] < br)) { bk = s_key[w]; br = s_row[w]; }
        cand_k[jj & 1] = bk;
        cand_r[jj & 1] = br;
      }
      __syncthreads();
      const int br = cand_r[jj & 1];
      if (tid < bw) {
        if (br < m) pub_p[jj & 1][tid] = P[(size_t)tid * rpc + (br - r0)];
        if (j >= r0 && j < r0 + nr) pub_j[jj & 1][tid] = P[(size_t)tid * rpc + (j - r0)];
      }
    }
    cl.sync();
    if (warp == 0) {   // the pivot (the same in every CTA) and rows p, j
      long long best = -1;
      int bi = m;
      if (lane < cs) {
        best = cl.map_shared_rank(cand_k, lane)[jj & 1];
        bi = cl.map_shared_rank(cand_r, lane)[jj & 1];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      const double bv = __longlong_as_double(best);
      const bool ok = bv > 0.0 && isfinite(bv) && bi < m;
      if (lane == 0) {
        s_fail = ok ? 0 : 1;
        s_p = bi;
      }
      if (ok && lane < bw) {
        const int op = bi / rpc, oj = j / rpc;
        rowp[lane] = cl.map_shared_rank(&pub_p[0][0], op)[(jj & 1) * GJB + lane];
        rowj[lane] = cl.map_shared_rank(&pub_j[0][0], oj)[(jj & 1) * GJB + lane];
      }
    }
    __syncthreads();
    if (s_fail) break;   // uniform over the cluster
    const int p = s_p;
    const S inv = S(1.0) / rowp[jj];
    if (tid < bw) newj[tid] = tid == jj ? inv : rowp[tid] * inv;
    if (q == 0 && tid == 0) piv[j] = p;
    __syncthreads();
    for (int rl = tid; rl < nr; rl += GJB_NT) {
      const int r = r0 + rl;
      if (r == j) {
        for (int c = 0; c < bw; ++c) P[(size_t)c * rpc + rl] = newj[c];
        continue;
      }
      const S mr = r == p ? rowj[jj] : colj[rl];
      for (int c = 0; c < bw; ++c) {
        S* pc = P + (size_t)c * rpc + rl;
        const S old = c == jj ? S(0.0) : (r == p ? rowj[c] : *pc);
        *pc = old - mr * newj[c];
      }
    }
    __syncthreads();
  }
  cl.sync();   // no CTA leaves while another may still read its row copies
  if (s_fail) {
    if (q == 0 && tid == 0) atomicOr(bad, 1);
    return;
  }
  for (int e = tid; e < bw * nr; e += GJB_NT) {
    const int c = e / nr, rl = e % nr;
    M[(r0 + rl) + (size_t)(c0 + c) * m] = P[(size_t)c * rpc + rl];
  }
}

// The panel's steps on cpb columns per CTA outside the panel [c0, c0 + bw):
// the row exchanges, then the rank-bw update with V read from the panel.
// Grid: boxes x apb column blocks.
template <class S, class Dims>
__global__ void __launch_bounds__(GJB_NT) k_gjb_apply(BigArgs g, S* ws, Dims dims, int c0, int cpb, int apb,
                                                      const int* bad) {
  extern __shared__ __align__(16) unsigned char ga_smem[];
  __shared__ int sp[GJB];
  int m;
  S *M, *pb_in, *pb_out;
  int* piv;
  dims(ws, g, blockIdx.x / apb, 0, m, M, pb_in, pb_out, piv);
  if (*bad || c0 >= m) return;
  const int bw = min(GJB, m - c0);
  const int q0 = (blockIdx.x % apb) * cpb;
  const int nc = min(cpb, m - bw - q0);
  if (nc <= 0) return;
  S* A = reinterpret_cast<S*>(ga_smem);   // nc columns, ld m
  const int tid = threadIdx.x;
  auto colof = [&](int cl) { const int q = q0 + cl; return q < c0 ? q : q + bw; };
  for (int e = tid; e < nc * m; e += GJB_NT) A[e] = M[(e % m) + (size_t)colof(e / m) * m];
  for (int i = tid; i < bw; i += GJB_NT) sp[i] = piv[c0 + i];
  __syncthreads();
  for (int cl = tid; cl < nc; cl += GJB_NT) {   // row exchanges in step order
    S* col = A + (size_t)cl * m;
    for (int i = 0; i < bw; ++i) {
      const int j = c0 + i, p = sp[i];
      if (p <= j || p >= m) continue;
      const S t = col[j];
      col[j] = col[p];
      col[p] = t;
    }
  }
  __syncthreads();
  const S* Pan = M + (size_t)c0 * m;
  for (int r = tid; r < m; r += GJB_NT) {
    S pr[GJB];
#pragma unroll
    for (int i = 0; i < GJB; ++i) pr[i] = i < bw ? Pan[r + (size_t)i * m] : S(0.0);
    const bool in_panel = r >= c0 && r < c0 + bw;
    for (int cl = 0; cl < nc; ++cl) {
      const S* col = A + (size_t)cl * m;
      S v = in_panel ? S(0.0) : col[r];
#pragma unroll
      for (int i = 0; i < GJB; ++i)
        if (i < bw) v += pr[i] * col[c0 + i];
      M[r + (size_t)colof(cl) * m] = v;
    }
  }
}

template <class S, class Dims>
__global__ void __launch_bounds__(BB_NT) k_bb_gj_step(BigArgs g, S* ws, Dims dims, int j, int ncb, int* bad) {
  bb_gj_body<S, Dims>(g, ws, dims, j, ncb, bad);
}

// All pivot steps in one cooperative launch, a grid barrier between steps.
// The same arithmetic as bb_gj_body, but each CTA keeps its BB_CB columns in
// shared memory for the whole inversion: per step it reads only the pivot
// column (written by that column's owner in the previous step) from global
// memory, and writes back its columns once at the end.
template <class S, class Dims>
__global__ void __launch_bounds__(BB_NT) k_bb_gj_coop(BigArgs g, S* ws, Dims dims, int nsteps, int ncb, int* bad,
                                                      GridBar gb) {
  extern __shared__ __align__(16) unsigned char bb_smem[];
  __shared__ int s_p;
  __shared__ double s_best;
  __shared__ S newj[BB_CB];
  const int b = blockIdx.x / ncb, cb = blockIdx.x % ncb;
  int m;
  S *M, *pb_in, *pb_out;
  int* piv;
  dims(ws, g, b, 0, m, M, pb_in, pb_out, piv);
  const int c_beg = cb * BB_CB, nc = max(0, min(m, c_beg + BB_CB) - c_beg);
  S* Ms = reinterpret_cast<S*>(bb_smem);   // own columns, [nc][m]
  S* pc = Ms + (size_t)BB_CB * m;          // pivot column of the step, [m]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < nc * m; e += BB_NT) Ms[e] = M[(size_t)c_beg * m + e];
  for (int j = 0; j < nsteps; ++j) {
    if (j < m && nc > 0) {
      dims(ws, g, b, j, m, M, pb_in, pb_out, piv);
      for (int r = tid; r < m; r += BB_NT) pc[r] = ldcg_s(pb_in + r);
      __syncthreads();
      if (warp == 0) {
        double best = -1.0;
        int bi = j;
        for (int r = j + lane; r < m; r += 32) {
          double v = abs2(pc[r]);
          if (v > best) { best = v; bi = r; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          double ob = __shfl_xor_sync(0xffffffffu, best, o);
          int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { s_p = bi; s_best = best; }
      }
      __syncthreads();
      if (!(s_best > 0.0) || !isfinite(s_best)) {
        if (tid == 0 && cb == 0) atomicOr(bad, 1);
      } else {
        const int p = s_p;
        if (tid == 0 && cb == 0) piv[j] = p;
        const S inv = S(1.0) / pc[p];
        for (int cl = tid; cl < nc; cl += BB_NT) {
          const int c = c_beg + cl;
          newj[cl] = c == j ? inv : Ms[(size_t)cl * m + p] * inv;   // row p moves to row j
        }
        __syncthreads();
        for (int e = tid; e < nc * m; e += BB_NT) {
          const int r = e % m, cl = e / m, c = c_beg + cl;
          if (r == j) continue;
          S* col = Ms + (size_t)cl * m;
          const S old = c == j ? S(0.0) : (r == p ? col[j] : col[r]);
          const S mr = pc[r == j ? p : (r == p ? j : r)];
          col[r] = old - mr * newj[cl];
        }
        __syncthreads();
        for (int cl = tid; cl < nc; cl += BB_NT) Ms[(size_t)cl * m + j] = newj[cl];
        __syncthreads();
        if (j + 1 >= c_beg && j + 1 < c_beg + nc)   // owner of the next pivot column publishes it
          for (int r = tid; r < m; r += BB_NT) pb_out[r] = Ms[(size_t)(j + 1 - c_beg) * m + r];
      }
    }
    if (!grid_sync(gb, (unsigned int)(j + 1) * gridDim.x)) return;
  }
  for (int e = tid; e < nc * m; e += BB_NT) M[(size_t)c_beg * m + e] = Ms[e];
}

// All pivot steps of one box in one thread-block cluster: the cluster's CTAs
// split the box's columns (cw each) and keep them in shared memory; per step
// the owner of the pivot column finds the pivot row and publishes the
// column's multipliers in its shared memory, one hardware cluster barrier
// later every CTA reads them over distributed shared memory and updates its
// own columns (the arithmetic of bb_gj_body).  The publication buffer
// alternates between two halves so one barrier per step suffices.  Shared
// layout per CTA: own columns [cw][m] | multipliers [m] | 2 x ([m] + inv, p).
template <class S, class Dims>
__global__ void __launch_bounds__(BB_NT) k_bb_gj_cluster(BigArgs g, S* ws, Dims dims, int nsteps, int cw, int* bad) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char bb_smem[];
  __shared__ int s_p;
  __shared__ double s_best;
  __shared__ S newj[64];
  const int crank = (int)cl.block_rank();
  const int b = blockIdx.x / (int)cl.num_blocks();
  int m;
  S *M, *pb_in, *pb_out;
  int* piv;
  dims(ws, g, b, 0, m, M, pb_in, pb_out, piv);
  const int c_beg = crank * cw, nc = max(0, min(m, c_beg + cw) - c_beg);
  S* Ms = reinterpret_cast<S*>(bb_smem);     // own columns
  S* ml = Ms + (size_t)cw * nsteps;          // this step's multipliers (local copy)
  S* pub = ml + nsteps;                      // 2 halves of nsteps + 2 scalars (inv, p)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < nc * m; e += BB_NT) Ms[e] = M[(size_t)c_beg * m + e];
  __syncthreads();
  bool failed = false;   // uniform over the cluster (every CTA reads the same published pivot)
  for (int j = 0; j < m; ++j) {
    const int owner = j / cw;
    S* half = pub + (size_t)(j & 1) * (nsteps + 2);
    if (crank == owner) {   // pivot search and publication
      const S* colj = Ms + (size_t)(j - c_beg) * m;
      if (warp == 0) {
        double best = -1.0;
        int bi = j;
        for (int r = j + lane; r < m; r += 32) {
          double v = abs2(colj[r]);
          if (v > best) { best = v; bi = r; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          double ob = __shfl_xor_sync(0xffffffffu, best, o);
          int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { s_p = bi; s_best = best; }
      }
      __syncthreads();
      const int p = s_p;
      const bool ok = s_best > 0.0 && isfinite(s_best);
      for (int r = tid; r < m; r += BB_NT) half[r] = colj[r == j ? p : (r == p ? j : r)];
      if (tid == 0) {
        half[nsteps] = ok ? S(1.0) / colj[p] : S(0.0);
        reinterpret_cast<int*>(half + nsteps + 1)[0] = ok ? p : -1;
        if (ok) piv[j] = p;
        else atomicOr(bad, 1);
      }
    }
    cl.sync();
    // multipliers, 1 / pivot and the pivot row from the owner's shared memory
    const S* rhalf = cl.map_shared_rank(half, owner);
    for (int r = tid; r < m; r += BB_NT) ml[r] = rhalf[r];
    const S inv = rhalf[nsteps];
    const int p = reinterpret_cast<const int*>(rhalf + nsteps + 1)[0];
    if (p < 0) failed = true;
    __syncthreads();
    if (!failed && nc > 0) {
      for (int q = tid; q < nc; q += BB_NT) {
        const int c = c_beg + q;
        newj[q] = c == j ? inv : Ms[(size_t)q * m + p] * inv;   // row p moves to row j
      }
      __syncthreads();
      for (int e = tid; e < nc * m; e += BB_NT) {
        const int r = e % m, q = e / m, c = c_beg + q;
        if (r == j) continue;
        S* col = Ms + (size_t)q * m;
        const S old = c == j ? S(0.0) : (r == p ? col[j] : col[r]);
        col[r] = old - ml[r] * newj[q];
      }
      __syncthreads();
      for (int q = tid; q < nc; q += BB_NT) Ms[(size_t)q * m + j] = newj[q];
      __syncthreads();
    }
  }
  cl.sync();   // no CTA leaves while another may still read its shared memory
  for (int e = tid; e < nc * m; e += BB_NT) M[(size_t)c_beg * m + e] = Ms[e];
}

// Final column order of a Gauss-Jordan inverse: position c holds column idx[c].
template <class S, class Dims>
__global__ void k_bb_unscramble(BigArgs g, S* ws, Dims dims, S* dst_base, int dst_kind, int ucb) {
  // grid: boxes x ucb column blocks of UNS_CB columns; shared: piv | idx (2 maxm ints)
  extern __shared__ int us_smem[];
  const int b = blockIdx.x / ucb, c0 = (blockIdx.x % ucb) * UNS_CB;
  int m;
  S *M, *pb_in, *pb_out;
  int* piv;
  dims(ws, g, b, 0, m, M, pb_in, pb_out, piv);
  if (c0 >= m) return;
  int* sp = us_smem;
  int* idx = us_smem + m;
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    sp[c] = piv[c];
    idx[c] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0)   // the row exchanges, last first, give the column order
    for (int j = m - 1; j >= 0; --j) {
      const int q = sp[j], t = idx[j];
      idx[j] = idx[q];
      idx[q] = t;
    }
  __syncthreads();
  S* dst = dims.dest(ws, g, b, dst_base, dst_kind);
  const int nc = min(UNS_CB, m - c0);
  for (int e = threadIdx.x; e < nc * m; e += blockDim.x) {
    const int r = e % m, c = c0 + e / m;
    dst[r + (size_t)c * m] = M[r + (size_t)idx[c] * m];
  }
}

// Accessors of the two inversions: D (n x n, A slot) and P X (k x k, Y slot).
struct DimsD {
  template <class S>
  __device__ void operator()(S* ws, const BigArgs& g, int b, int j, int& m, S*& M, S*& pin, S*& pout,
                             int*& piv) const {
    const int n = g.n[b], k = g.k[b];
    S* A = ws + g.bo[b];
    m = n;
    M = A;
    S* buf = A + 2 * (size_t)n * n + (size_t)n * k + (size_t)k * k;
    pin = buf + (size_t)(j & 1) * n;
    pout = buf + (size_t)((j + 1) & 1) * n;
    piv = reinterpret_cast<int*>(buf + 2 * (size_t)n);
  }
  template <class S>
  __device__ S* dest(S* ws, const BigArgs& g, int b, S*, int) const {
    const int n = g.n[b];
    return ws + g.bo[b] + (size_t)n * n;   // Dinv slot
  }
};
struct DimsY {
  const int64_t* lamoff;
  template <class S>
  __device__ void operator()(S* ws, const BigArgs& g, int b, int j, int& m, S*& M, S*& pin, S*& pout,
                             int*& piv) const {
    const int n = g.n[b], k = g.k[b];
    S* A = ws + g.bo[b];
    m = k;
    M = A + 2 * (size_t)n * n + (size_t)n * k;
    S* buf = A + 2 * (size_t)n * n + (size_t)n * k + (size_t)k * k;
    pin = buf + (size_t)(j & 1) * n;
    pout = buf + (size_t)((j + 1) & 1) * n;
    piv = reinterpret_cast<int*>(buf + 2 * (size_t)n);
  }
  template <class S>
  __device__ S* dest(S* ws, const BigArgs& g, int b, S* lam, int) const {
    return lam + lamoff[b];
  }
};

// X = Dinv P^T (column i per CTA), and its sk rows combined into Y = P X
// (both from global memory).
template <class S>
__global__ void k_bb_X(FaArgs a, BigArgs g, const S* Tpool, S* ws, int maxk) {
  const int b = blockIdx.x / maxk, i = blockIdx.x % maxk;
  const int n = g.n[b], k = g.k[b], nr = n - k;
  if (i >= k) return;
  const int* lp = a.lperm + a.off[b];
  const S* T = Tpool + a.toff[b];
  S* A = ws + g.bo[b];
  const S* Dinv = A + (size_t)n * n;
  S* X = A + 2 * (size_t)n * n;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    S s = Dinv[r + (size_t)lp[i] * n];
    for (int q = 0; q < nr; ++q) s += T[i + (size_t)q * k] * Dinv[r + (size_t)lp[k + q] * n];
    X[r + (size_t)i * n] = s;
  }
}

template <class S>
__global__ void k_bb_Y(FaArgs a, BigArgs g, const S* Tpool, S* ws, int maxk) {
  const int b = blockIdx.x / maxk, c = blockIdx.x % maxk;
  const int n = g.n[b], k = g.k[b], nr = n - k;
  if (c >= k) return;
  const int* lp = a.lperm + a.off[b];
  const S* T = Tpool + a.toff[b];
  S* A = ws + g.bo[b];
  const S* X = A + 2 * (size_t)n * n;
  S* Y = A + 2 * (size_t)n * n + (size_t)n * k;
  S* buf = Y + (size_t)k * k;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    S s = X[lp[i] + (size_t)c * n];
    for (int q = 0; q < nr; ++q) s += T[i + (size_t)q * k] * X[lp[k + q] + (size_t)c * n];
    Y[i + (size_t)c * k] = s;
    if (c == 0) buf[i] = s;   // first pivot column of the Lambda inversion
  }
}

// calL = X Lambda, calR = Lambda X^T, calD = Dinv - calL X^T (column c per CTA).
template <class S>
__global__ void k_bb_products(FaArgs a, BigArgs g, S* ws, const S* Lampool, S* Upool, S* Lpool, int maxn) {
  const int b = blockIdx.x / maxn, c = blockIdx.x % maxn;
  const int n = g.n[b], k = g.k[b];
  if (c >= n) return;
  S* A = ws + g.bo[b];
  const S* Dinv = A + (size_t)n * n;
  const S* X = A + 2 * (size_t)n * n;
  const S* Lam = Lampool + a.lamoff[b];
  S* U = Upool + a.uoff[b];
  S* Lf = Lpool + a.loff[b];
  const int ldu = n + k;
  if (c < k)
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      S s = S(0.0);
      for (int q = 0; q < k; ++q) s += X[r + (size_t)q * n] * Lam[q + (size_t)c * k];
      Lf[r + (size_t)c * n] = s;
    }
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    S s = S(0.0);
    for (int q = 0; q < k; ++q) s += Lam[i + (size_t)q * k] * X[c + (size_t)q * n];
    U[n + i + (size_t)c * ldu] = s;
  }
  // calD[:, c] = Dinv[:, c] - X Lambda X[c, :]^T: w = Lambda X[c, :]^T first
  extern __shared__ __align__(16) unsigned char bp_smem[];
  S* w = reinterpret_cast<S*>(bp_smem);   // k entries
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    S s = S(0.0);
    for (int q = 0; q < k; ++q) s += Lam[i + (size_t)q * k] * X[c + (size_t)q * n];
    w[i] = s;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    S s = Dinv[r + (size_t)c * n];
    for (int q = 0; q < k; ++q) s -= X[r + (size_t)q * n] * w[q];
    U[r + (size_t)c * ldu] = s;
  }
}

// Skeleton ids of every box into the parent depth's active vector.
__global__ void k_emit(const int* n, const int* k, const int64_t* off, const int64_t* skoff, const int* act,
                       const int* lperm, int nbox, int* act_up, int* owner_up) {
  int b = blockIdx.x;
  if (b >= nbox) return;
  int kb = k[b];
  for (int i = threadIdx.x; i < kb; i += blockDim.x) {
    act_up[skoff[b] + i] = act[off[b] + lperm[off[b] + i]];
    owner_up[skoff[b] + i] = b;
  }
}

template <class S>
__global__ void k_to_float(const S* in, typename lowp<S>::type* out, int64_t cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) out[i] = typename lowp<S>::type(in[i]);
}

// ------------------------------------------------------------- host helpers
// Flops of k_factor for one box: Gauss-Jordan on [D | I] (3 n^3), X = D^-1 P^T,
// P X, Gauss-Jordan on [P X | I] (3 k^3), calL, calR, calD.
double factor_flops(double n, double k) {
  double nr = n - k;
  return 3.0 * n * n * n + 2.0 * n * k * nr + 2.0 * k * k * nr + 3.0 * k * k * k + 4.0 * n * k * k +
         2.0 * n * n * k;
}
// Algorithmic flops of the column-pivoted QR of an m x n block stopped at
// rank k (Householder QR with downdated norms: 4mnk - 2k^2(m + n) + 4k^3/3)
// and of T = R11^-1 R12 by back substitution (k^2 (n - k)).  The m n kernel
// evaluations of the fill are not counted as flops.
double id_flops(double m, double n, double k) {
  return 4.0 * m * n * k - 2.0 * k * k * (m + n) + 4.0 * k * k * k / 3.0 + k * k * (n - k);
}

template <class T>
int upload(Handle* h, T** d, const std::vector<T>& v, cudaStream_t st) {
  RS_TRY(dalloc_t(h, d, std::max<size_t>(1, v.size())));
  if (!v.empty()) RS_CUDA(cudaMemcpyAsync(*d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
  return RS_OK;
}

size_t scal_bytes(const Handle* h) { return h->cplx ? sizeof(c128) : sizeof(double); }

Geo make_geo(const Handle* h, int depth) {
  Geo g;
  for (int d = 0; d < 3; ++d) g.lower[d] = h->center[d] - h->half;
  g.side = (2.0 * h->half) / (double)(1ll << depth);
  g.dim = h->dim;
  g.nproxy = h->nproxy;
  g.ratio = h->ratio;
  g.constrow = 0;
  if (h->kp.kind == RS_LAPLACE2D) {
    double rho = h->ratio * (std::sqrt(2.0) / 2.0) * g.side;
    g.constrow = std::fabs(std::log(rho)) < 0.1 ? 1 : 0;
  }
  // the double layer's row ID always has the constant row (the column ID
  // fills it with zeros, so both sides share one row count)
  if (h->kp.kind == RS_LAPLACE2D_DL) g.constrow = 1;
  return g;
}

Pts make_pts(const Handle* h) {
  Pts p;
  p.x = h->pts;
  p.y = h->pts + h->N;
  p.z = h->dim == 3 ? h->pts + 2 * h->N : nullptr;
  p.nx = h->dlg;
  p.ny = h->dlg ? h->dlg + h->N : nullptr;
  p.kap = h->dlg ? h->dlg + 2 * h->N : nullptr;
  return p;
}

// Largest dynamic shared memory a CTA may opt into (minus room for the
// kernels' static shared variables).
int max_dyn_smem() {
  static const int v = [] {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      cudaGetLastError();
      return 200 * 1024;
    }
    return optin - 4096;
  }();
  return v;
}

int num_sms() {
  static const int v = [] {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return 132;
    }
    return nsm;
  }();
  return v;
}

// Whether `grid` CTAs of `kern` can all be resident at once (the condition
// of a cooperative launch).
bool coop_fits(const void* kern, int grid, int nt, size_t smem) {
  int dev = 0, nsm = 0, occ = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nt, smem)) {
    cudaGetLastError();
    return false;
  }
  return coop && grid <= occ * nsm;
}

// Arrival counter of a grid barrier (zeroed, stream ordered); `flag` is the
// status word set when a wait gives up.
int make_bar(GridBar* gb, int* flag, cudaStream_t st) {
  RS_CUDA(cudaMallocAsync((void**)&gb->count, sizeof(unsigned int), st));
  RS_CUDA(cudaMemsetAsync(gb->count, 0, sizeof(unsigned int), st));
  gb->flag = flag;
  return RS_OK;
}

// Cluster launch of nb boxes, one cluster of cs CTAs per box, each CTA with
// cw = ceil(width / cs) columns.  Picks cs from {16, 8, 4, 2} to minimise
// waves x (cw + 4): the co-resident cluster count comes from the occupancy
// API (clusters of 16 CTAs are few per GPC), the 4 stands for the fixed
// per-step cost of the barriers.  Returns false when no size fits.
template <class Kern, class SmemOf>
bool pick_cluster(Kern kern, int nb, int width, int nt, SmemOf smem_of, cudaStream_t st, int* cs_out, int* cw_out,
                  size_t* smem_out) {
  double best = 0.0;
  bool found = false;
  for (int cs : {16, 8, 4, 2}) {
    const int cw = div_up(width, cs);
    const size_t smem = smem_of(cw);
    if (smem > (size_t)max_dyn_smem()) continue;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        (cs > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb * cs);
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess || ncl < 1) {
      cudaGetLastError();
      continue;
    }
    const double cost = (double)div_up(nb, ncl) * (cw + 4);
    if (!found || cost < best) {
      found = true;
      best = cost;
      *cs_out = cs;
      *cw_out = cw;
      *smem_out = smem;
    }
  }
  if (found) {   // leave the chosen size's attribute set
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem_out) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
  }
  return found;
}

template <class Kern, class... Args>
int launch_cluster(Kern kern, int nb, int cs, int nt, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nb * cs);
  cfg.blockDim = dim3(nt);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  RS_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
  RS_CHECK_LAUNCH();
  return RS_OK;
}

// Randomized ID on the multi-CTA path: column c of box b of the sample
// Y = Omega M (l_b rows, compact with leading dimension l_b) from the filled
// M (m_b rows, g.m / g.moff); boxes with l_b == m_b are copied.  The column's
// squared norm and the box's rank bound are reset for the sample.
template <class S>
__global__ void __launch_bounds__(BI_NT) k_sketch_big(const double* sketch, BigId g, const int* n, const int* l,
                                                      const int64_t* yoff, const S* Mws, S* Yws, int maxn) {
  const int b = blockIdx.x / maxn, c = blockIdx.x % maxn;
  if (c >= n[b]) return;
  const int mb = g.m[b], lb = l[b];
  const S* col = Mws + g.moff[b] + (size_t)c * mb;
  S* out = Yws + yoff[b] + (size_t)c * lb;
  double s2 = 0.0;
  for (int i = threadIdx.x; i < lb; i += BI_NT) {
    S acc = S(0.0);
    if (lb == mb) {
      acc = col[i];
    } else {
      for (int r = 0; r < mb; ++r) acc += scal(col[r], sketch[i + (size_t)r * SKETCH_STRIDE]);
    }
    out[i] = acc;
    s2 += abs2(acc);
  }
  __shared__ double red[BI_NT];
  red[threadIdx.x] = s2;
  __syncthreads();
  for (int o = BI_NT / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    g.nrm[g.noff[b] + c] = red[0];
    if (c == 0) g.kk[b] = min(lb, n[b]);
  }
}

template <class S>
int run_id_big(Handle* h, Level& lv, IdArgs a, const std::vector<int>& mrows_in, cudaStream_t st) {
  std::vector<int> mrows = mrows_in;
  const int nb = lv.nbox;
  std::vector<int64_t> moff(nb), noff(nb);
  int64_t macc = 0, nacc = 0;
  int maxkmax = 0;
  for (int b = 0; b < nb; ++b) {
    moff[b] = macc;
    noff[b] = nacc;
    macc += (int64_t)mrows[b] * lv.h_n[b];
    nacc += lv.h_n[b];
    maxkmax = std::max(maxkmax, std::min(mrows[b], lv.h_n[b]));
  }
  BigId g{};
  int64_t *dmo, *dno;
  RS_TRY(upload(h, &dmo, moff, st));
  RS_TRY(upload(h, &dno, noff, st));
  g.m = a.mrows;
  g.n = a.n;
  g.moff = dmo;
  g.noff = dno;
  S* Mws = nullptr;
  RS_CUDA(cudaMallocAsync((void**)&Mws, sizeof(S) * std::max<int64_t>(1, macc), st));
  g.ntot = std::max<int64_t>(1, nacc);
  RS_CUDA(cudaMallocAsync((void**)&g.nrm, sizeof(double) * 2 * g.ntot, st));
  RS_CUDA(cudaMallocAsync((void**)&g.map0, sizeof(int) * std::max<int64_t>(1, nacc), st));
  RS_CUDA(cudaMallocAsync((void**)&g.map1, sizeof(int) * std::max<int64_t>(1, nacc), st));
  RS_CUDA(cudaMallocAsync((void**)&g.r00, sizeof(double) * nb, st));
  RS_CUDA(cudaMallocAsync((void**)&g.kk, sizeof(int) * nb, st));
  RS_CUDA(cudaMallocAsync(&g.rdiag, sizeof(S) * std::max<int64_t>(1, nacc), st));
  const int maxn = lv.maxn;
  prof_begin(P_ID, st);
  k_bbid_fill<S><<<nb * maxn, BI_NT, 0, st>>>(a, g, Mws, maxn);
  RS_CHECK_LAUNCH();
  if (a.sketch_p > 0) {   // randomized ID: the QR below runs on the samples
    std::vector<int> lrows(nb);
    std::vector<int64_t> yoff(nb);
    int64_t yacc = 0;
    int lmax = 0;
    for (int b = 0; b < nb; ++b) {
      lrows[b] = mrows[b] > lv.h_n[b] + a.sketch_p ? lv.h_n[b] + a.sketch_p : mrows[b];
      yoff[b] = yacc;
      yacc += (int64_t)lrows[b] * lv.h_n[b];
      lmax = std::max(lmax, lrows[b]);
    }
    int *dl;
    int64_t* dyo;
    RS_TRY(upload(h, &dl, lrows, st));
    RS_TRY(upload(h, &dyo, yoff, st));
    S* Yws = nullptr;
    RS_CUDA(cudaMallocAsync((void**)&Yws, sizeof(S) * std::max<int64_t>(1, yacc), st));
    k_sketch_big<S><<<nb * maxn, BI_NT, 0, st>>>(a.sketch, g, a.n, dl, dyo, Mws, Yws, maxn);
    RS_CHECK_LAUNCH();
    RS_CUDA(cudaFreeAsync(Mws, st));
    Mws = Yws;
    mrows = lrows;
    g.m = dl;
    g.moff = dyo;
    a.mrows = dl;
    a.mmax = lmax;
    maxkmax = 0;
    for (int b = 0; b < nb; ++b) maxkmax = std::max(maxkmax, std::min(lrows[b], lv.h_n[b]));
  }
  const int ncb = div_up(maxn, BI_CB);
  const size_t id_smem = sizeof(S) * (size_t)a.mmax + sizeof(int) * (size_t)a.nmax;
  RS_CUDA(cudaFuncSetAttribute(k_bbid_step<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)id_smem));
  // first choice: one thread-block cluster per box, its columns resident in
  // the CTAs' shared memory
  bool coop_done = false;
  {
    int cs = 0, cw = 0;
    size_t smem = 0;
    auto smem_of = [&](int w) {
      return sizeof(S) * ((size_t)w * a.mmax + a.mmax + 2) + sizeof(double) * ((size_t)w + 2) +
             sizeof(int) * ((size_t)a.nmax + w + 2);
    };
    if (!(path_force() & PF_ID_NOCLUSTER) &&
        pick_cluster(k_bbid_cluster<S>, nb, maxn, BI_NT, smem_of, st, &cs, &cw, &smem)) {
      RS_TRY(launch_cluster(k_bbid_cluster<S>, nb, cs, BI_NT, smem, st, a, g, Mws, cw, a.lperm));
      path_count(PATH_ID_CLUSTER);
      coop_done = true;
    }
  }
  // else a cooperative launch: CB columns per CTA (8 first; then 16 or 32 when
  // the grid is too large to be resident at once, 4 or 2 when the column
  // cache is too large for shared memory)
  auto try_coop = [&](auto cbc) -> int {
    constexpr int CB = decltype(cbc)::value;
    if (coop_done || (path_force() & PF_ID_NOCOOP)) return RS_OK;
    const int ncbc = div_up(maxn, CB);
    const size_t co_smem = ((id_smem + 15) & ~(size_t)15) + sizeof(S) * (size_t)CB * a.mmax;
    if (co_smem > (size_t)max_dyn_smem()) return RS_OK;
    RS_CUDA(cudaFuncSetAttribute(k_bbid_coop<S, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)co_smem));
    if (!coop_fits((const void*)k_bbid_coop<S, CB>, nb * ncbc, BI_NT, co_smem)) return RS_OK;
    GridBar gb{};
    RS_TRY(make_bar(&gb, h->status + 1, st));
    int nsteps = maxkmax, ncbv = ncbc, nbv = nb;
    int* lp = a.lperm;
    void* args[] = {&a, &g, &Mws, &nsteps, &ncbv, &nbv, &lp, &gb};
    RS_CUDA(cudaLaunchCooperativeKernel((const void*)k_bbid_coop<S, CB>, dim3(nb * ncbc), dim3(BI_NT), args, co_smem,
                                        st));
    RS_CHECK_LAUNCH();
    RS_CUDA(cudaFreeAsync(gb.count, st));
    path_count(PATH_ID_COOP);
    coop_done = true;
    return RS_OK;
  };
  RS_TRY(try_coop(std::integral_constant<int, 8>{}));
  RS_TRY(try_coop(std::integral_constant<int, 16>{}));   // fewer CTAs when the grid does not fit
  RS_TRY(try_coop(std::integral_constant<int, 32>{}));
  RS_TRY(try_coop(std::integral_constant<int, 4>{}));    // less shared memory per CTA
  RS_TRY(try_coop(std::integral_constant<int, 2>{}));
  if (!coop_done) {
    // one launch per step; every 8 steps, stop early once every box of the
    // level has found its rank
    int* d_active = nullptr;
    int h_active = 1;
    path_count(PATH_ID_STEP);
    RS_CUDA(cudaMallocAsync((void**)&d_active, sizeof(int), st));
    for (int j = 0; j < maxkmax; ++j) {
      k_bbid_step<S><<<nb * ncb, BI_NT, id_smem, st>>>(a, g, Mws, j, ncb, a.lperm);
      RS_CHECK_LAUNCH();
      if ((j & 7) == 7 && j + 1 < maxkmax) {
        k_bbid_active<<<1, 256, 0, st>>>(g, a.n, nb, j + 1, d_active);
        RS_CHECK_LAUNCH();
        RS_CUDA(cudaMemcpyAsync(&h_active, d_active, sizeof(int), cudaMemcpyDeviceToHost, st));
        RS_CUDA(cudaStreamSynchronize(st));
        if (!h_active) break;
      }
    }
    RS_CUDA(cudaFreeAsync(d_active, st));
  }
  const int wpb = BI_NT / 32;
  const int tb = div_up(maxn, wpb);
  k_bbid_T<S><<<nb * tb, BI_NT, 0, st>>>(a, g, Mws, (S*)lv.T, tb);
  RS_CHECK_LAUNCH();
  prof_end(P_ID, st, 0.0, 0.0);
  for (void* q : {(void*)Mws, (void*)g.nrm, (void*)g.map0, (void*)g.map1, (void*)g.r00, (void*)g.kk, g.rdiag})
    RS_CUDA(cudaFreeAsync(q, st));
  return RS_OK;
}

template <class S>
int run_id(Handle* h, Level& lv, const IdArgs& a0, const std::vector<int>& mrows, int64_t msum, S* Tout,
           cudaStream_t st) {
  IdArgs a = a0;
  size_t sb = sizeof(S);
  size_t extra = (size_t)a.mmax * sb + 2 * (size_t)a.nmax * sizeof(double) + 3 * (size_t)a.geo.nproxy * sizeof(double) +
                 (size_t)a.mmax * sizeof(int64_t) + (size_t)a.nmax * sizeof(int) + 2 * (size_t)a.mmax * sizeof(int) + 64;
  int64_t mnmax = 0;
  for (int b = 0; b < lv.nbox; ++b) mnmax = std::max<int64_t>(mnmax, (int64_t)mrows[b] * lv.h_n[b]);
  a.mnmax = mnmax;
  size_t mbytes = (size_t)mnmax * sb;
  const size_t limit = (size_t)max_dyn_smem();
  S* Mws = nullptr;
  a.smem_path = (mbytes + extra <= limit) ? 1 : 0;
  // boxes too large for one CTA: several CTAs per box
  // (non-symmetric kernels keep one CTA per box, with M in global memory
  // when it does not fit shared memory)
  const bool big_ok = !h->nonsym && a.geo.nproxy <= 256 &&
                      sizeof(S) * (size_t)a.mmax + sizeof(int) * (size_t)a.nmax <= 200 * 1024;
  if (big_ok && (!a.smem_path || (path_force() & PF_ID_BIG))) return run_id_big<S>(h, lv, a, mrows, st);
  size_t smem = a.smem_path ? mbytes + extra : extra;
  if (smem > 227 * 1024) return fail(RS_ERR_ARG, "box too large for shared staging (m=%d n=%d)", a.mmax, a.nmax);
  if (!a.smem_path) {
    std::vector<int64_t> moff(lv.nbox);
    int64_t acc = 0;
    for (int b = 0; b < lv.nbox; ++b) { moff[b] = acc; acc += (int64_t)mrows[b] * lv.h_n[b]; }
    int64_t* dmoff;
    RS_TRY(upload(h, &dmoff, moff, st));
    a.moff = dmoff;
    RS_CUDA(cudaMallocAsync((void**)&Mws, sb * std::max<int64_t>(1, acc), st));
  }
  RS_CUDA(cudaFuncSetAttribute(k_id<S, ID_NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // near-field blocks of every colleague pair, evaluated once (the kernels
  // are symmetric: G(x, y) = G(y, x))
  std::vector<int> pi, pj;
  std::vector<int64_t> pbase, slot_base((size_t)lv.nbox * 27, -1);
  int64_t pacc = 0;
  for (int i = 0; i < lv.nbox; ++i)
    for (int si = 0; si < lv.h_ncoll[i]; ++si) {
      const int j = lv.h_coll[(size_t)i * 27 + si];
      if (j <= i) continue;
      pi.push_back(i);
      pj.push_back(j);
      pbase.push_back(pacc);
      slot_base[(size_t)i * 27 + si] = pacc;
      for (int sj = 0; sj < lv.h_ncoll[j]; ++sj)
        if (lv.h_coll[(size_t)j * 27 + sj] == i) slot_base[(size_t)j * 27 + sj] = pacc;
      pacc += (int64_t)lv.h_n[i] * lv.h_n[j];
    }
  S* pairs = nullptr;
  prof_begin(P_ID, st);
  if (!pi.empty() && !h->nonsym) {
    int *dpi, *dpj;
    int64_t *dpb, *dsb;
    RS_TRY(upload(h, &dpi, pi, st));
    RS_TRY(upload(h, &dpj, pj, st));
    RS_TRY(upload(h, &dpb, pbase, st));
    RS_TRY(upload(h, &dsb, slot_base, st));
    RS_CUDA(cudaMallocAsync((void**)&pairs, sb * (size_t)pacc, st));
    k_near_pairs<S><<<(unsigned)pi.size(), 128, 0, st>>>(a.kp, a.pts, a.n, a.off, a.act, dpi, dpj, dpb, pairs);
    RS_CHECK_LAUNCH();
    a.pair_base = dsb;
    a.pairs = pairs;
  }
  k_id<S, ID_NT><<<lv.nbox, ID_NT, smem, st>>>(a, Mws, Tout);
  RS_CHECK_LAUNCH();
  path_count(PATH_ID_CTA);
  prof_end(P_ID, st, 0.0, 0.0);
  if (Mws) RS_CUDA(cudaFreeAsync(Mws, st));
  if (pairs) RS_CUDA(cudaFreeAsync(pairs, st));
  (void)msum;
  return RS_OK;
}

// The Gauss-Jordan steps of every box on one thread-block cluster per box:
// cs CTAs with cw = ceil(nsteps / cs) <= 64 columns each, when their shared
// memory fits (cs from pick_cluster); *done = false if no cluster shape fits.
template <class S, class Dims>
int run_gj_cluster(BigArgs g, S* ws, Dims dims, int nsteps, int nb, int* bad, cudaStream_t st, bool* done) {
  *done = false;
  int cs = 0, cw = 0;
  size_t smem = 0;
  auto smem_of = [&](int w) -> size_t {
    if (w > 64) return ~(size_t)0;   // k_bb_gj_cluster keeps at most 64 columns' multipliers
    return sizeof(S) * ((size_t)w * nsteps + nsteps + 2 * ((size_t)nsteps + 2));
  };
  if (!pick_cluster(k_bb_gj_cluster<S, Dims>, nb, nsteps, BB_NT, smem_of, st, &cs, &cw, &smem)) return RS_OK;
  RS_TRY(launch_cluster(k_bb_gj_cluster<S, Dims>, nb, cs, BB_NT, smem, st, g, ws, dims, nsteps, cw, bad));
  path_count(PATH_GJ_CLUSTER);
  *done = true;
  return RS_OK;
}

// The nsteps in-place Gauss-Jordan steps of every box of a level: a cluster
// per box when the columns fit; else (the root, or boxes too large for a
// cluster) the blocked form; else one cooperative launch when the grid is
// resident at once, else one launch per step.
template <class S, class Dims>
int run_gj_steps(Handle* h, BigArgs g, S* ws, Dims dims, int nsteps, int nb, int ncb, size_t smem, int* bad,
                 cudaStream_t st) {
  const int force = path_force();
  if (nb >= 2 && !(force & PF_GJ_NOCLUSTER)) {   // one cluster per box when the columns fit
    bool done = false;
    RS_TRY((run_gj_cluster<S, Dims>(g, ws, dims, nsteps, nb, bad, st, &done)));
    if (done) return RS_OK;
  }
  if (nsteps >= 128 && !(force & PF_GJ_NOBLOCKED)) {   // the root, or boxes too large for a cluster: blocked
    const int m = nsteps;   // the largest box
    path_count(PATH_GJ_BLOCKED);
    // panel steps on a cluster per box (rows split over its CTAs), else one CTA
    int pcs = 0, prpc = 0;
    size_t pc_smem = 0;
    {
      auto smem_of = [&](int rows) { return sizeof(S) * (size_t)rows * GJB; };
      int cw = 0;
      if (pick_cluster(k_gjb_panel_cl<S, Dims>, nb, m, GJB_NT, smem_of, st, &pcs, &cw, &pc_smem)) prpc = cw;
    }
    const size_t psmem = sizeof(S) * (size_t)m * (GJB + 1);
    const int in_smem = psmem <= (size_t)max_dyn_smem() ? 1 : 0;
    const size_t pa_smem = in_smem ? psmem : sizeof(S) * (size_t)m;
    RS_CUDA(cudaFuncSetAttribute(k_gjb_panel<S, Dims>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pa_smem));
    // columns per CTA: enough CTAs for two per SM, within shared memory
    const int nout = m - std::min(GJB, m);
    int cpb = std::max(1, nb * nout / (2 * num_sms()));
    cpb = std::min(cpb, std::min(GJB_APPLY_MAXC, (int)((size_t)max_dyn_smem() / (sizeof(S) * (size_t)m))));
    if (cpb < 1) return fail(RS_ERR_ARG, "root block too large for the blocked inversion (m=%d)", m);
    const size_t ap_smem = sizeof(S) * (size_t)m * cpb;
    RS_CUDA(cudaFuncSetAttribute(k_gjb_apply<S, Dims>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ap_smem));
    for (int c0 = 0; c0 < m; c0 += GJB) {
      if (prpc > 0) {
        RS_TRY(launch_cluster(k_gjb_panel_cl<S, Dims>, nb, pcs, GJB_NT, pc_smem, st, g, ws, dims, c0, prpc, bad));
      } else {
        k_gjb_panel<S, Dims><<<nb, GJB_NT, pa_smem, st>>>(g, ws, dims, c0, in_smem, bad);
        RS_CHECK_LAUNCH();
      }
      const int no = m - std::min(GJB, m - c0);
      if (no > 0) {
        const int apb = div_up(no, cpb);
        k_gjb_apply<S, Dims><<<nb * apb, GJB_NT, ap_smem, st>>>(g, ws, dims, c0, cpb, apb, bad);
        RS_CHECK_LAUNCH();
      }
    }
    return RS_OK;
  }
  const size_t csmem = sizeof(S) * (size_t)(BB_CB + 1) * nsteps;   // own columns + pivot column (m <= nsteps)
  const bool co_ok = csmem <= (size_t)max_dyn_smem();
  if (co_ok)
    RS_CUDA(cudaFuncSetAttribute(k_bb_gj_coop<S, Dims>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem));
  if (co_ok && !(force & PF_GJ_NOCOOP) && coop_fits((const void*)k_bb_gj_coop<S, Dims>, nb * ncb, BB_NT, csmem)) {
    path_count(PATH_GJ_COOP);
    GridBar gb{};
    RS_TRY(make_bar(&gb, bad + 1, st));   // the status word after the singularity flag
    void* args[] = {&g, &ws, &dims, &nsteps, &ncb, &bad, &gb};
    RS_CUDA(cudaLaunchCooperativeKernel((const void*)k_bb_gj_coop<S, Dims>, dim3(nb * ncb), dim3(BB_NT), args, csmem,
                                        st));
    RS_CHECK_LAUNCH();
    RS_CUDA(cudaFreeAsync(gb.count, st));
    return RS_OK;
  }
  RS_CUDA(cudaFuncSetAttribute(k_bb_gj_step<S, Dims>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  path_count(PATH_GJ_STEP);
  for (int j = 0; j < nsteps; ++j) {
    k_bb_gj_step<S, Dims><<<nb * ncb, BB_NT, smem, st>>>(g, ws, dims, j, ncb, bad);
    RS_CHECK_LAUNCH();
  }
  return RS_OK;
}

// Big boxes (few of them, or too large for one CTA's shared memory): several
// CTAs per box -- assembly, the two Gauss-Jordan inversions (run_gj_steps:
// clusters, blocked for the root and the largest boxes, cooperative or
// per-step launches as fallbacks) and the products.
template <class S>
int run_factor_big(Handle* h, Level& lv, FaArgs a, const Level* child, double by, cudaStream_t st) {
  const int nb = lv.nbox;
  std::vector<int64_t> bo(nb);
  int64_t acc = 0;
  int maxk = 1;
  for (int b = 0; b < nb; ++b) {
    int64_t n = lv.h_n[b], k = lv.h_k[b];
    bo[b] = acc;
    acc += 2 * n * n + n * k + k * k + 2 * n + n;   // A | Dinv | X | Y | pivot buffers | pivots
    maxk = std::max<int>(maxk, (int)k);
  }
  BigArgs g{};
  g.n_box = nb;
  g.n = lv.n;
  g.k = lv.k;
  int64_t* dbo;
  RS_TRY(upload(h, &dbo, bo, st));
  g.bo = dbo;
  S* ws = nullptr;
  const int maxn = lv.maxn;
  RS_CUDA(cudaMallocAsync((void**)&ws, sizeof(S) * std::max<int64_t>(1, acc), st));
  const S* cL = child ? (const S*)child->Lam : nullptr;
  double fl = 0.0;
  for (int b = 0; b < nb; ++b) {
    double n = lv.h_n[b], k = lv.h_k[b];
    fl += factor_flops(n, k) - n * n * n - k * k * k;
  }
  if (is_cplx<S>::value) fl *= 4.0;
  prof_begin(P_FACTOR, st);
  k_bb_assemble<S><<<nb * maxn, BB_NT, 0, st>>>(a, g, cL, ws, maxn);
  RS_CHECK_LAUNCH();
  const int ncb = div_up(maxn, BB_CB);
  const size_t gj_smem = sizeof(S) * (size_t)maxn;
  RS_TRY((run_gj_steps<S, DimsD>(h, g, ws, DimsD{}, maxn, nb, ncb, gj_smem, a.bad, st)));
  const int ucb = div_up(maxn, UNS_CB);
  const size_t us_smem = 2 * sizeof(int) * (size_t)maxn;
  k_bb_unscramble<S, DimsD><<<nb * ucb, BB_NT, us_smem, st>>>(g, ws, DimsD{}, (S*)nullptr, 0, ucb);
  RS_CHECK_LAUNCH();
  if (lv.maxk > 0) {
    k_bb_X<S><<<nb * maxk, BB_NT, 0, st>>>(a, g, (const S*)lv.T, ws, maxk);
    RS_CHECK_LAUNCH();
    k_bb_Y<S><<<nb * maxk, BB_NT, 0, st>>>(a, g, (const S*)lv.T, ws, maxk);
    RS_CHECK_LAUNCH();
    const int nck = div_up(maxk, BB_CB);
    DimsY dy{lv.lamoff};
    const size_t gy_smem = sizeof(S) * (size_t)maxk;
    RS_TRY((run_gj_steps<S, DimsY>(h, g, ws, dy, maxk, nb, nck, gy_smem, a.bad, st)));
    k_bb_unscramble<S, DimsY><<<nb * ucb, BB_NT, us_smem, st>>>(g, ws, dy, (S*)lv.Lam, 1, ucb);
    RS_CHECK_LAUNCH();
  }
  const size_t pr_smem = sizeof(S) * (size_t)std::max(1, maxk);
  RS_CUDA(cudaFuncSetAttribute(k_bb_products<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pr_smem));
  k_bb_products<S><<<nb * maxn, BB_NT, pr_smem, st>>>(a, g, ws, (const S*)lv.Lam, (S*)lv.U, (S*)lv.Lf, maxn);
  RS_CHECK_LAUNCH();
  prof_end(P_FACTOR, st, by, fl);
  RS_CUDA(cudaFreeAsync(ws, st));
  return RS_OK;
}

template <class S>
int run_factor(Handle* h, Level& lv, FaArgs a, const Level* child, cudaStream_t st) {
  // workspace: [D | I] (2 n^2) + X (n k) + [PX | I] (2 k^2) (+ P D^-1 (k n),
  // non-symmetric kernels)
  std::vector<int64_t> wsoff(lv.nbox);
  int64_t acc = 0;
  for (int b = 0; b < lv.nbox; ++b) {
    int64_t n = lv.h_n[b], k = lv.h_k[b];
    wsoff[b] = acc;
    acc += 2 * n * n + n * k + 2 * k * k + (h->nonsym ? k * n : 0);
  }
  // shared-memory path when every box's D, X and Lambda fit
  size_t sm_need = 0;
  for (int b = 0; b < lv.nbox; ++b) {
    size_t n = lv.h_n[b], k = lv.h_k[b];
    sm_need = std::max(sm_need, sizeof(S) * (n * n + n * k + k * k + n) + sizeof(int) * n + 16);
  }
  // one CTA per box in shared memory when the boxes fit and are enough to
  // spread over the SMs; a few large boxes take several CTAs each
  const bool few = 2 * lv.nbox < num_sms() && lv.maxn >= 64 && sizeof(S) * (size_t)lv.maxn <= 200 * 1024;
  // (non-symmetric kernels: the general one-CTA-per-box elimination below)
  const bool smem_path = sm_need <= 200 * 1024 && !few && !(path_force() & PF_FACTOR_BIG) && !h->nonsym;
  double fl0 = 0.0, by0 = 0.0;
  for (int b = 0; b < lv.nbox; ++b) {
    double n = lv.h_n[b], k = lv.h_k[b];
    fl0 += factor_flops(n, k) - (smem_path ? n * n * n + k * k * k : 0.0);   // in-place GJ: n^3 MACs
    by0 += (double)sizeof(S) * ((n + k) * n + n * k + k * k);
  }
  if (is_cplx<S>::value) fl0 *= 4.0;
  if (smem_path) {
    const S* cL = child ? (const S*)child->Lam : nullptr;
    prof_begin(P_FACTOR, st);
    RS_CUDA(cudaFuncSetAttribute(k_factor_smem<S, FA_SM_NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm_need));
    k_factor_smem<S, FA_SM_NT><<<lv.nbox, FA_SM_NT, sm_need, st>>>(a, (const S*)lv.T, cL, (S*)lv.U, (S*)lv.Lf,
                                                                    (S*)lv.Lam);
    RS_CHECK_LAUNCH();
    path_count(PATH_FAC_SMEM);
    prof_end(P_FACTOR, st, by0, fl0);
    return RS_OK;
  }
  if (sizeof(S) * (size_t)lv.maxn <= 200 * 1024 && !h->nonsym) {
    path_count(PATH_FAC_BIG);
    return run_factor_big<S>(h, lv, a, child, by0, st);
  }
  path_count(PATH_FAC_GENERIC);
  int64_t* dws;
  RS_TRY(upload(h, &dws, wsoff, st));
  a.wsoff = dws;
  S* ws = nullptr;
  RS_CUDA(cudaMallocAsync((void**)&ws, sizeof(S) * std::max<int64_t>(1, acc), st));
  size_t smem = sizeof(S) * std::max(1, lv.maxn);
  RS_CUDA(cudaFuncSetAttribute(k_factor<S, FA_NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  double fl = 0.0, by = 0.0;
  for (int b = 0; b < lv.nbox; ++b) {
    double n = lv.h_n[b], k = lv.h_k[b];
    fl += factor_flops(n, k);
    by += (double)sizeof(S) * ((n + k) * n + n * k + k * k);   // factors written
  }
  if (is_cplx<S>::value) fl *= 4.0;
  prof_begin(P_FACTOR, st);
  k_factor<S, FA_NT><<<lv.nbox, FA_NT, smem, st>>>(a, (const S*)lv.T, child ? (const S*)child->Lam : nullptr, ws,
                                                   (S*)lv.U, (S*)lv.Lf, (S*)lv.Lam);
  RS_CHECK_LAUNCH();
  prof_end(P_FACTOR, st, by, fl);
  RS_CUDA(cudaFreeAsync(ws, st));
  return RS_OK;
}

// Status words: [0] a singular or non-finite pivot, [1] a grid barrier gave
// up, both in the skeletonization (checked per depth with the ranks); [2],
// [3] the same in the factorization (which runs on its own stream and is
// checked once at the end).

// Sizes and offsets of the factor pools of a level (host), then allocate.
int alloc_factors(Handle* h, Level& lv, cudaStream_t st) {
  std::vector<int64_t> uoff(lv.nbox), loff(lv.nbox), lamoff(lv.nbox);
  int64_t us = 0, ls = 0, lams = 0;
  for (int b = 0; b < lv.nbox; ++b) {
    int64_t n = lv.h_n[b], k = lv.h_k[b];
    uoff[b] = us; us += (n + k) * n;
    loff[b] = ls; ls += n * k;
    lamoff[b] = lams; lams += k * k;
  }
  lv.usz = us; lv.lsz = ls; lv.lamsz = lams;
  lv.h_uoff = uoff;
  lv.h_loff = loff;
  RS_TRY(upload(h, &lv.uoff, uoff, st));
  RS_TRY(upload(h, &lv.loff, loff, st));
  RS_TRY(upload(h, &lv.lamoff, lamoff, st));
  size_t sb = scal_bytes(h);
  RS_TRY(dalloc(h, &lv.U, sb * std::max<int64_t>(1, us)));
  RS_TRY(dalloc(h, &lv.Lf, sb * std::max<int64_t>(1, ls)));
  RS_TRY(dalloc(h, &lv.Lam, sb * std::max<int64_t>(1, lams)));
  {   // forward-operator factors of the refinement residual (fwd2.cu): float
      // and double-float (real), complex float and complex double-float (complex)
    const size_t lo = h->cplx ? sizeof(c64) : sizeof(float), hi = h->cplx ? sizeof(cdfloat) : sizeof(dfloat);
    RS_TRY(dalloc(h, &lv.FU32, lo * std::max<int64_t>(1, us)));
    RS_TRY(dalloc(h, &lv.FUdf, hi * std::max<int64_t>(1, us)));
    RS_TRY(dalloc(h, &lv.FL32, lo * std::max<int64_t>(1, ls)));
    RS_TRY(dalloc(h, &lv.FLdf, hi * std::max<int64_t>(1, ls)));
  }
  h->factor_scalars += us + ls;
  return RS_OK;
}

// fs waits for the work queued on st so far.
int follow(cudaStream_t fs, cudaStream_t st) {
  cudaEvent_t ev;
  RS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(ev, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(fs, ev, 0);
  cudaEventDestroy(ev);
  if (e != cudaSuccess) return fail(RS_ERR_CUDA, "stream ordering: %s", cudaGetErrorString(e));
  return RS_OK;
}

}  // namespace

int check_factor_status(Handle* h, cudaStream_t st) {
  int bad[2] = {0, 0};
  RS_CUDA(cudaMemcpyAsync(bad, h->status + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  RS_CUDA(cudaStreamSynchronize(st));
  if (bad[1]) return fail(RS_ERR_TIMEOUT, "rs_build: a grid barrier wait ran out during factorization");
  if (bad[0]) return fail(RS_ERR_SINGULAR, "rs_build: singular block during factorization");
  return RS_OK;
}

namespace {

// The factorization of one depth (or the root, k = 0) on fs, after the
// skeletonization work queued on st.
int factor_level(Handle* h, Level& lv, const Level* child, const int* lperm, const int64_t* toff, bool leaf,
                 cudaStream_t st, cudaStream_t fs, const int* lperm_r = nullptr) {
  FaArgs f{};
  f.kp = h->kp;
  f.pts = make_pts(h);
  f.leaf_level = leaf;
  f.n = lv.n;
  f.k = lv.k;
  f.off = lv.off;
  f.act = lv.act;
  f.owner = lv.owner;
  if (child) {
    f.cskoff = child->skoff;
    f.ck = child->k;
    f.clamoff = child->lamoff;
  }
  f.lperm = lperm;
  f.toff = toff;
  f.uoff = lv.uoff;
  f.loff = lv.loff;
  f.lamoff = lv.lamoff;
  f.bad = h->status + 2;
  f.fu32 = (float*)lv.FU32;
  f.fudf = (dfloat*)lv.FUdf;
  if (h->nonsym) {
    f.general = 1;
    f.act_r = lv.act_r;
    f.lperm_r = lperm_r ? lperm_r : lperm;
    f.Tr = lv.T_r ? lv.T_r : lv.T;
  }
  RS_TRY(follow(fs, st));
  if (h->cplx) RS_TRY(run_factor<c128>(h, lv, f, child, fs));
  else RS_TRY(run_factor<double>(h, lv, f, child, fs));
  return RS_OK;
}

}  // namespace

// Skeletonize every box of depth `depth` (1 <= depth <= L) on st and queue
// its factorization on fs; fills the active sets of depth-1.
int skeletonize_level(Handle* h, int depth, cudaStream_t st, cudaStream_t fs) {
  Level& lv = h->lv[depth];
  const int nbox = lv.nbox;
  // active sets of the leaves come from the tree
  if (depth == h->L) {
    lv.h_n.resize(nbox);
    std::vector<int64_t> off(nbox);
    for (int b = 0; b < nbox; ++b) {
      int e = b + 1 < nbox ? lv.h_begin[b + 1] : (int)h->N;
      lv.h_n[b] = e - lv.h_begin[b];
      off[b] = lv.h_begin[b];
    }
    lv.ntot = h->N;
    lv.h_off = off;
    RS_TRY(upload(h, &lv.n, lv.h_n, st));
    RS_TRY(upload(h, &lv.off, off, st));
  }
  lv.maxn = 0;
  for (int b = 0; b < nbox; ++b) lv.maxn = std::max(lv.maxn, lv.h_n[b]);

  Geo geo = make_geo(h, depth);
  std::vector<int> mrows(nbox);
  std::vector<int64_t> toff(nbox);
  int64_t tacc = 0, msum = 0;
  lv.maxm = 0;
  for (int b = 0; b < nbox; ++b) {
    int near = 0;
    for (int j = 0; j < lv.h_ncoll[b]; ++j) near += lv.h_n[lv.h_coll[(size_t)b * 27 + j]];
    mrows[b] = near + h->nproxy + geo.constrow;
    lv.maxm = std::max(lv.maxm, mrows[b]);
    msum += (int64_t)mrows[b] * lv.h_n[b];
    toff[b] = tacc;
    int64_t n = lv.h_n[b];
    tacc += (n * n) / 4;
  }
  lv.tsz = tacc;
  int* dm;
  RS_TRY(upload(h, &dm, mrows, st));
  RS_TRY(upload(h, &lv.toff, toff, st));
  size_t sb = scal_bytes(h);
  RS_TRY(dalloc(h, &lv.T, sb * std::max<int64_t>(1, tacc)));
  RS_TRY(dalloc_t(h, &lv.k, nbox));
  RS_TRY(dalloc_t(h, &lv.lperm, std::max<int64_t>(1, lv.ntot)));
  int* krow = nullptr;   // non-symmetric kernels: the row IDs' ranks
  if (h->nonsym) {
    if (!lv.act_r) lv.act_r = lv.act;   // the leaves: rows and columns are the same points
    RS_TRY(dalloc(h, &lv.T_r, sb * std::max<int64_t>(1, tacc)));
    RS_TRY(dalloc_t(h, &lv.lperm_r, std::max<int64_t>(1, lv.ntot)));
    RS_TRY(dalloc_t(h, &krow, nbox));
  } else {
    lv.act_r = lv.act;
    lv.lperm_r = lv.lperm;
    lv.T_r = lv.T;
  }

  IdArgs a{};
  a.kp = h->kp;
  a.pts = make_pts(h);
  a.geo = geo;
  a.eps = h->eps;
  a.n = lv.n;
  a.off = lv.off;
  a.act = lv.act;
  a.act_near = lv.act_r;
  a.row_side = 0;
  a.kmin = nullptr;
  a.ncoll = lv.ncoll;
  a.coll = lv.coll;
  a.coords = lv.coords;
  a.mrows = dm;
  a.toff = lv.toff;
  a.kout = lv.k;
  a.lperm = lv.lperm;
  a.mmax = lv.maxm;
  a.nmax = lv.maxn;
  a.qr_df = h->id_df && !h->cplx;
  a.sketch_p = 0;
  a.sketch = nullptr;
  if (h->id_p > 0) {   // randomized ID: the sketch table for this depth's largest m
    if (lv.maxn + h->id_p > SKETCH_STRIDE)
      return fail(RS_ERR_ARG, "rs_build: randomized ID needs n + oversampling <= %d (n = %d)", SKETCH_STRIDE, lv.maxn);
    if (h->sketch_m < lv.maxm) {
      const int64_t cnt = (int64_t)SKETCH_STRIDE * lv.maxm;
      RS_TRY(dalloc(h, (void**)&h->sketch, sizeof(double) * cnt));
      k_sketch_table<<<std::max<int64_t>(1, std::min<int64_t>(4096, (cnt + 255) / 256)), 256, 0, st>>>(h->id_seed, cnt,
                                                                                                    h->sketch);
      RS_CHECK_LAUNCH();
      h->sketch_m = lv.maxm;
    }
    a.sketch = h->sketch;
    a.sketch_p = h->id_p;
  }
  if (h->cplx) RS_TRY(run_id<c128>(h, lv, a, mrows, msum, (c128*)lv.T, st));
  else RS_TRY(run_id<double>(h, lv, a, mrows, msum, (double*)lv.T, st));
  if (h->nonsym) {
    // Two-sided compression (Sec. 3.1): the row ID of every box (the
    // transposed block row against the colleagues' column points and the
    // proxy charges) at no less than the column rank, then the column ID
    // again at no less than the row rank, so both sides end at
    // max(row rank, column rank).
    IdArgs ar = a;
    ar.act = lv.act_r;
    ar.act_near = lv.act;
    ar.row_side = 1;
    ar.kmin = lv.k;
    ar.kout = krow;
    ar.lperm = lv.lperm_r;
    RS_TRY(run_id<double>(h, lv, ar, mrows, msum, (double*)lv.T_r, st));
    IdArgs ac = a;
    ac.kmin = krow;
    RS_TRY(run_id<double>(h, lv, ac, mrows, msum, (double*)lv.T, st));
  }

  // ranks -> skeleton offsets in the parent depth (one synchronisation for
  // the ranks and the skeletonization's status words)
  lv.h_k.resize(nbox);
  int bad[2] = {0, 0};
  std::vector<int> hkr(h->nonsym ? nbox : 0);
  RS_CUDA(cudaMemcpyAsync(lv.h_k.data(), lv.k, sizeof(int) * nbox, cudaMemcpyDeviceToHost, st));
  if (h->nonsym) RS_CUDA(cudaMemcpyAsync(hkr.data(), krow, sizeof(int) * nbox, cudaMemcpyDeviceToHost, st));
  RS_CUDA(cudaMemcpyAsync(bad, h->status, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  RS_CUDA(cudaStreamSynchronize(st));
  if (bad[1]) return fail(RS_ERR_TIMEOUT, "rs_build: a grid barrier wait ran out during skeletonization");
  if (bad[0]) return fail(RS_ERR_SINGULAR, "rs_build: singular block during skeletonization");
  for (int b = 0; b < (int)hkr.size(); ++b)
    if (hkr[b] != lv.h_k[b])
      return fail(RS_ERR_SINGULAR, "rs_build: box %d of depth %d: row rank %d and column rank %d differ", b, depth,
                  hkr[b], lv.h_k[b]);
  if (prof_on()) {
    double fl = 0.0, by = 0.0;
    for (int b = 0; b < nbox; ++b) {
      fl += id_flops(mrows[b], lv.h_n[b], lv.h_k[b]);
      by += (double)sb * (double)lv.h_k[b] * (lv.h_n[b] - lv.h_k[b]);   // T written
    }
    prof_amend(P_ID, by, h->cplx ? 4.0 * fl : fl);
  }
  std::vector<int64_t> skoff(nbox);
  int64_t kacc = 0;
  lv.maxk = 0;
  for (int b = 0; b < nbox; ++b) {
    skoff[b] = kacc;
    kacc += lv.h_k[b];
    lv.maxk = std::max(lv.maxk, lv.h_k[b]);
  }
  lv.ksum = kacc;
  lv.h_skoff = skoff;
  RS_TRY(upload(h, &lv.skoff, skoff, st));

  // factor (on fs, overlapping the next depths' skeletonization)
  RS_TRY(alloc_factors(h, lv, st));
  const Level* child = depth < h->L ? &h->lv[depth + 1] : nullptr;
  RS_TRY(factor_level(h, lv, child, lv.lperm, lv.toff, depth == h->L, st, fs, lv.lperm_r));

  // active sets of depth-1: skeletons of the children, in child order
  Level& up = h->lv[depth - 1];
  up.ntot = kacc;
  RS_TRY(dalloc_t(h, &up.act, std::max<int64_t>(1, kacc)));
  RS_TRY(dalloc_t(h, &up.owner, std::max<int64_t>(1, kacc)));
  k_emit<<<nbox, 64, 0, st>>>(lv.n, lv.k, lv.off, lv.skoff, lv.act, lv.lperm, nbox, up.act, up.owner);
  RS_CHECK_LAUNCH();
  if (h->nonsym) {   // the row active sets of depth-1: the children's row skeletons
    RS_TRY(dalloc_t(h, &up.act_r, std::max<int64_t>(1, kacc)));
    k_emit<<<nbox, 64, 0, st>>>(lv.n, lv.k, lv.off, lv.skoff, lv.act_r, lv.lperm_r, nbox, up.act_r, up.owner);
    RS_CHECK_LAUNCH();
  } else {
    up.act_r = up.act;
  }
  up.h_n.assign(up.nbox, 0);
  std::vector<int64_t> upoff(up.nbox, -1);
  for (int b = 0; b < nbox; ++b) {
    int p = lv.h_parent[b];
    if (upoff[p] < 0) upoff[p] = skoff[b];
    up.h_n[p] += lv.h_k[b];
  }
  up.h_off = upoff;
  RS_TRY(upload(h, &up.n, up.h_n, st));
  RS_TRY(upload(h, &up.off, upoff, st));
  return RS_OK;
}

// Root: calS assembled like any upper-level block (or A itself when the tree
// has a single box), inverted densely.
int factor_root(Handle* h, cudaStream_t st, cudaStream_t fs) {
  Level& lv = h->lv[0];
  if (h->L == 0) {
    lv.h_n.assign(1, (int)h->N);
    lv.ntot = h->N;
    std::vector<int64_t> off(1, 0);
    lv.h_off = off;
    RS_TRY(upload(h, &lv.n, lv.h_n, st));
    RS_TRY(upload(h, &lv.off, off, st));
  }
  lv.maxn = lv.h_n[0];
  if (!lv.act_r) lv.act_r = lv.act;
  lv.h_k.assign(1, 0);
  std::vector<int> k0(1, 0);
  RS_TRY(upload(h, &lv.k, k0, st));
  RS_TRY(alloc_factors(h, lv, st));
  const Level* child = h->L > 0 ? &h->lv[1] : nullptr;
  int* dummy_perm;
  RS_TRY(dalloc_t(h, &dummy_perm, std::max<int64_t>(1, lv.ntot)));
  return factor_level(h, lv, child, dummy_perm, nullptr, h->L == 0, st, fs);
}

int make_fp32_copies(Handle* h, cudaStream_t st) {
  prof_begin(P_COPY32, st);
  double by = 0.0;
  for (int d = 0; d <= h->L; ++d) {
    Level& lv = h->lv[d];
    size_t lb = h->cplx ? sizeof(c64) : sizeof(float);
    RS_TRY(dalloc(h, &lv.U32, lb * std::max<int64_t>(1, lv.usz)));
    RS_TRY(dalloc(h, &lv.Lf32, lb * std::max<int64_t>(1, lv.lsz)));
    if (h->cplx) {
      if (lv.usz) k_to_float<c128><<<div_up(lv.usz, 256), 256, 0, st>>>((c128*)lv.U, (c64*)lv.U32, lv.usz);
      if (lv.lsz) k_to_float<c128><<<div_up(lv.lsz, 256), 256, 0, st>>>((c128*)lv.Lf, (c64*)lv.Lf32, lv.lsz);
    } else {
      if (lv.usz) k_to_float<double><<<div_up(lv.usz, 256), 256, 0, st>>>((double*)lv.U, (float*)lv.U32, lv.usz);
      if (lv.lsz) k_to_float<double><<<div_up(lv.lsz, 256), 256, 0, st>>>((double*)lv.Lf, (float*)lv.Lf32, lv.lsz);
    }
    RS_CHECK_LAUNCH();
    by += (double)(lv.usz + lv.lsz) * (scal_bytes(h) + lb);
  }
  prof_end(P_COPY32, st, by, 0.0);
  return RS_OK;
}

}  // namespace rs
