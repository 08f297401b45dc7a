// Solve phase and forward operator.
//
// Solve (eq. multilevel-inverse applied right to left, Sec. 4.3): vectors
// are kept per tree depth in "point-major" layout v[pos * R + col] so that
// every box's block of rows is one contiguous chunk.
//   upward   for depth L..1:  [u_i ; c_i] = [calD_i ; calR_i] b_i, c_i lands
//            in the parent's active vector at skoff_i
//   root     x_0 = calS^-1 c (the root's U holds calS^-1, k = 0)
//   downward for depth 1..L:  x_i = u_i + calL_i x_parent[skoff_i ...]
// Forward operator A_RS (eq. multilevel-compression, Sec. 3.3), FP64 (the
// rs_matvec path, an independent check of the refinement's residual):
//   upward   z_parent[skoff_i + a] = (P_i z_i)[a] = z_i[sk_a] + sum_e T[a,e] z_i[rd_e]
//            y_i = D^(l)_i z_i with the kernel block evaluated on the fly from
//            the coordinates (leaf: A(I_i, I_i); above: w G between skeletons
//            of different children, zero within one child; root: same form)
//   downward y_i += P_i^T y_parent[skoff_i ...]
#include <algorithm>
#include <mutex>
#include <vector>

#include "rs_internal.h"

namespace rs {

namespace {

constexpr int SV_NT = 256;

template <class S> struct hi_of { using type = double; };
template <> struct hi_of<c64> { using type = c128; };
template <> struct hi_of<c128> { using type = c128; };

template <class D, class S> __device__ inline D cvt(S v) { return D(v); }
template <> __device__ inline float cvt<float, double>(double v) { return (float)v; }
template <> __device__ inline double cvt<double, float>(float v) { return (double)v; }
template <> __device__ inline c64 cvt<c64, c128>(c128 v) { return c64((float)v.re, (float)v.im); }
template <> __device__ inline c128 cvt<c128, c64>(c64 v) { return c128((double)v.re, (double)v.im); }

// out[i*R + c] = B[perm[i] + c*ldb]  (caller order -> tree order)
template <class SI, class S>
__global__ void k_perm_in(const SI* B, int64_t ldb, const int* perm, int64_t N, int R, S* out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * R) return;
  int64_t i = e / R;
  int c = (int)(e % R);
  out[e] = cvt<S, SI>(B[perm[i] + (int64_t)c * ldb]);
}

// X[perm[i] + c*ldx] = in[i*R + c]
template <class S, class SO>
__global__ void k_perm_out(const S* in, const int* perm, int64_t N, int R, SO* X, int64_t ldx) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * R) return;
  int64_t i = e / R;
  int c = (int)(e % R);
  X[perm[i] + (int64_t)c * ldx] = cvt<SO, S>(in[e]);
}

struct BoxView {
  const int* n;
  const int* k;
  const int64_t* off;
  const int64_t* skoff;
};

// Upward step of one depth: [u ; c] = U b per box.  One CTA per
// (box, column tile of CT columns).  b is staged in shared memory when it
// fits (STAGE), otherwise read through L1.
template <class S, int CT, bool STAGE>
__global__ void __launch_bounds__(SV_NT) k_up(BoxView bv, const int64_t* uoff, const S* U, const S* vin, S* uout,
                                             S* cout, int R, int ntile) {
  extern __shared__ __align__(16) unsigned char smem[];
  S* vs = reinterpret_cast<S*>(smem);
  const int b = blockIdx.x / ntile, tile = blockIdx.x % ntile;
  const int c0 = tile * CT, cw = min(CT, R - c0);
  const int n = bv.n[b], k = bv.k[b], rows = n + k;
  const int64_t off = bv.off[b];
  const int64_t sk = bv.skoff ? bv.skoff[b] : 0;
  if (STAGE) {
    for (int e = threadIdx.x; e < n * cw; e += SV_NT) {
      int q = e / cw, c = e % cw;
      vs[q * CT + c] = vin[(off + q) * R + c0 + c];
    }
    __syncthreads();
  }
  auto V = [&](int q, int c) -> S { return STAGE ? vs[q * CT + c] : vin[(off + q) * R + c0 + c]; };
  const S* Ub = U + uoff[b];
  if (CT == 1) {
    for (int r = threadIdx.x; r < rows; r += SV_NT) {
      S s0 = S(0.0), s1 = S(0.0), s2 = S(0.0), s3 = S(0.0);
      int q = 0;
      for (; q + 4 <= n; q += 4) {
        s0 += Ub[r + (size_t)q * rows] * V(q, 0);
        s1 += Ub[r + (size_t)(q + 1) * rows] * V(q + 1, 0);
        s2 += Ub[r + (size_t)(q + 2) * rows] * V(q + 2, 0);
        s3 += Ub[r + (size_t)(q + 3) * rows] * V(q + 3, 0);
      }
      for (; q < n; ++q) s0 += Ub[r + (size_t)q * rows] * V(q, 0);
      S s = (s0 + s1) + (s2 + s3);
      if (r < n) uout[off + r] = s;
      else cout[sk + (r - n)] = s;
    }
  } else {
    for (int e = threadIdx.x; e < rows * cw; e += SV_NT) {
      int r = e / cw, c = e % cw;
      S s = S(0.0);
#pragma unroll 4
      for (int q = 0; q < n; ++q) s += Ub[r + (size_t)q * rows] * V(q, c);
      if (r < n) uout[(off + r) * R + c0 + c] = s;
      else cout[(sk + (r - n)) * R + c0 + c] = s;
    }
  }
}

// Downward step: x = u + calL x_parent, in place on u.
template <class S, int CT, bool STAGE>
__global__ void __launch_bounds__(SV_NT) k_down(BoxView bv, const int64_t* loff, const S* Lf, const S* xpar, S* u,
                                               int R, int ntile) {
  extern __shared__ __align__(16) unsigned char smem[];
  S* xs = reinterpret_cast<S*>(smem);
  const int b = blockIdx.x / ntile, tile = blockIdx.x % ntile;
  const int c0 = tile * CT, cw = min(CT, R - c0);
  const int n = bv.n[b], k = bv.k[b];
  const int64_t off = bv.off[b], sk = bv.skoff[b];
  if (STAGE) {
    for (int e = threadIdx.x; e < k * cw; e += SV_NT) {
      int q = e / cw, c = e % cw;
      xs[q * CT + c] = xpar[(sk + q) * R + c0 + c];
    }
    __syncthreads();
  }
  auto XP = [&](int q, int c) -> S { return STAGE ? xs[q * CT + c] : xpar[(sk + q) * R + c0 + c]; };
  const S* Lb = Lf + loff[b];
  if (CT == 1) {
    for (int r = threadIdx.x; r < n; r += SV_NT) {
      S s0 = u[off + r], s1 = S(0.0), s2 = S(0.0), s3 = S(0.0);
      int q = 0;
      for (; q + 3 <= k; q += 3) {
        s1 += Lb[r + (size_t)q * n] * XP(q, 0);
        s2 += Lb[r + (size_t)(q + 1) * n] * XP(q + 1, 0);
        s3 += Lb[r + (size_t)(q + 2) * n] * XP(q + 2, 0);
      }
      for (; q < k; ++q) s1 += Lb[r + (size_t)q * n] * XP(q, 0);
      u[off + r] = s0 + (s1 + (s2 + s3));
    }
  } else {
    for (int e = threadIdx.x; e < n * cw; e += SV_NT) {
      int r = e / cw, c = e % cw;
      S s = S(0.0);
#pragma unroll 4
      for (int q = 0; q < k; ++q) s += Lb[r + (size_t)q * n] * XP(q, c);
      int64_t idx = (off + r) * R + c0 + c;
      u[idx] = u[idx] + s;
    }
  }
}

// ---------------------------------------------------------- forward operator
struct FwdView {
  const int* n;
  const int* k;
  const int64_t* off;
  const int64_t* skoff;
  const int* act;
  const int* owner;
  const int* lperm;
  const int64_t* toff;
  int leaf_level;
  const int* act_r;     // row active set (targets; = act for symmetric kernels)
  const int* lperm_r;   // row ID's column order (= lperm for symmetric kernels)
};

// z_parent[skoff + a] = z[sk_a] + sum_e T[a, e] z[rd_e]
template <class S>
__global__ void k_fwd_proj(FwdView fv, const S* T, const S* z, S* zpar, int R) {
  const int b = blockIdx.x;
  const int n = fv.n[b], k = fv.k[b], nr = n - k;
  const int64_t off = fv.off[b], sk = fv.skoff[b];
  const int* lp = fv.lperm + off;
  const S* Tb = T + fv.toff[b];
  for (int e = threadIdx.x; e < k * R; e += blockDim.x) {
    int a = e / R, c = e % R;
    S s = z[(off + lp[a]) * R + c];
    for (int q = 0; q < nr; ++q) s += Tb[a + (size_t)q * k] * z[(off + lp[k + q]) * R + c];
    zpar[(sk + a) * R + c] = s;
  }
}

// y_i = D_i z_i with kernel entries from the coordinates.  CTA per
// (box, row tile of 64, column tile of 32); kernel block chunks of 32 columns
// are staged in shared memory.
constexpr int FD_RT = 64, FD_CT = 32, FD_GC = 32;
template <class S>
__global__ void __launch_bounds__(SV_NT) k_fwd_dblock(FwdView fv, KParams kp, Pts pts, const S* z, S* y, int R,
                                                     int nrt, int nct) {
  constexpr int GC = sizeof(S) > 8 ? FD_GC / 2 : FD_GC;   // keep static smem under 48 KB
  __shared__ S G[GC][FD_RT + 1];
  __shared__ S zs[GC][FD_CT];
  const int b = blockIdx.x / (nrt * nct);
  const int rt = (blockIdx.x / nct) % nrt, ct = blockIdx.x % nct;
  const int n = fv.n[b];
  const int r0 = rt * FD_RT, c0 = ct * FD_CT;
  if (r0 >= n || c0 >= R) return;
  const int rw = min(FD_RT, n - r0), cw = min(FD_CT, R - c0);
  const int64_t off = fv.off[b];
  constexpr int PER = FD_RT * FD_CT / SV_NT;  // outputs per thread
  S acc[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) acc[i] = S(0.0);
  for (int g0 = 0; g0 < n; g0 += GC) {
    const int gw = min(GC, n - g0);
    for (int e = threadIdx.x; e < GC * FD_RT; e += SV_NT) {
      int r = e % FD_RT, q = e / FD_RT;
      S v = S(0.0);
      if (r < rw && q < gw) {
        int pr = off + r0 + r, pq = off + g0 + q;
        int ir = fv.act_r[pr], iq = fv.act[pq];
        if (fv.leaf_level) v = system_entry<S>(kp, pts, ir, iq);
        else if (fv.owner[pr] != fv.owner[pq]) v = offdiag_entry<S>(kp, pts, ir, iq);
      }
      G[q][r] = v;
    }
    for (int e = threadIdx.x; e < GC * FD_CT; e += SV_NT) {
      int q = e / FD_CT, c = e % FD_CT;
      zs[q][c] = (q < gw && c < cw) ? z[(off + g0 + q) * R + c0 + c] : S(0.0);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      int e = threadIdx.x + i * SV_NT;
      int r = e / FD_CT, c = e % FD_CT;
      S s = acc[i];
      for (int q = 0; q < gw; ++q) s += G[q][r] * zs[q][c];
      acc[i] = s;
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    int e = threadIdx.x + i * SV_NT;
    int r = e / FD_CT, c = e % FD_CT;
    if (r < rw && c < cw) y[(off + r0 + r) * R + c0 + c] = acc[i];
  }
}

// y[sk_a] += w[a], y[rd_e] += sum_a T[a, e] w[a],  w = y_parent[skoff ...]
// (the row ID's order and T: L_i = Q_i^T)
template <class S>
__global__ void k_fwd_down(FwdView fv, const S* T, const S* ypar, S* y, int R) {
  const int b = blockIdx.x;
  const int n = fv.n[b], k = fv.k[b];
  const int64_t off = fv.off[b], sk = fv.skoff[b];
  const int* lp = fv.lperm_r + off;
  const S* Tb = T + fv.toff[b];
  for (int e = threadIdx.x; e < n * R; e += blockDim.x) {
    int t = e / R, c = e % R;
    S s;
    if (t < k) {
      s = ypar[(sk + t) * R + c];
    } else {
      int q = t - k;
      s = S(0.0);
      for (int a = 0; a < k; ++a) s += Tb[a + (size_t)q * k] * ypar[(sk + a) * R + c];
    }
    int64_t idx = (off + lp[t]) * R + c;
    y[idx] = y[idx] + s;
  }
}

// out[c] = sum_i |v[i + c*N]|^2, one block per column (fixed order).
template <class S>
__global__ void k_colnorm2(const S* v, int64_t N, double* out) {
  __shared__ double s[SV_NT];
  const S* col = v + (int64_t)blockIdx.x * N;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += SV_NT) acc += abs2(col[i]);
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = SV_NT / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = s[0];
}

template <class S>
__global__ void k_axpy(S* x, const S* d, int64_t cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) x[i] = x[i] + d[i];
}

// ------------------------------------------------------------------- host
size_t sbytes(bool cplx, int prec) {
  if (prec == RS_PREC_FP64) return cplx ? sizeof(c128) : sizeof(double);
  if (prec == MODE_FWD_DF) return cplx ? sizeof(cdfloat) : sizeof(dfloat);
  return cplx ? sizeof(c64) : sizeof(float);
}

int ensure_work(Handle* h, int prec, int R, cudaStream_t st) {
  Handle::Work& w = h->work[prec];
  if (w.R >= R && w.prec == prec) return RS_OK;
  // grow: free the old buffers (stream ordered)
  for (void* p : w.v) if (p) RS_CUDA(cudaFreeAsync(p, st));
  for (void* p : w.u) if (p) RS_CUDA(cudaFreeAsync(p, st));
  w.v.assign(h->L + 1, nullptr);
  w.u.assign(h->L + 1, nullptr);
  size_t sb = sbytes(h->cplx, prec);
  w.bytes = 0;
  for (int d = 0; d <= h->L; ++d) {
    size_t cnt = (size_t)std::max<int64_t>(1, h->lv[d].ntot) * R;
    RS_CUDA(cudaMallocAsync(&w.v[d], cnt * sb, st));
    RS_CUDA(cudaMallocAsync(&w.u[d], cnt * sb, st));
    w.bytes += 2 * cnt * sb;
  }
  w.R = R;
  w.prec = prec;
  ++w.gen;
  return RS_OK;
}

BoxView box_view(const Level& lv) { return BoxView{lv.n, lv.k, lv.off, lv.skoff}; }

template <class S, class SIO>
int solve_impl(Handle* h, int prec, const SIO* B, int64_t ldb, int R, SIO* X, int64_t ldx, cudaStream_t st) {
  RS_TRY(ensure_work(h, prec, R, st));
  Handle::Work& w = h->work[prec];
  const int64_t N = h->N;
  const int L = h->L;
  int nb = div_up(N * R, 256);
  const double sS = sizeof(S), sIO = sizeof(SIO), cf = is_cplx<S>::value ? 4.0 : 1.0;
  prof_begin(P_PERM, st);
  k_perm_in<SIO, S><<<nb, 256, 0, st>>>(B, ldb, h->perm, N, R, (S*)w.v[L]);
  RS_CHECK_LAUNCH();
  prof_end(P_PERM, st, (double)N * R * (sS + sIO) + 4.0 * N, 0.0);
  const int CT = R == 1 ? 1 : 32;
  const int ntile = div_up(R, CT);
  const size_t stage_limit = 96 * 1024;
  for (int d = L; d >= 0; --d) {
    const Level& lv = h->lv[d];
    const S* U = (const S*)(prec == RS_PREC_FP64 ? lv.U : lv.U32);
    S* cout = d > 0 ? (S*)w.v[d - 1] : nullptr;
    size_t smem = sizeof(S) * (size_t)std::max(1, lv.maxn) * CT;
    BoxView bv = box_view(lv);
    if (d == 0) bv.skoff = nullptr;
    const S* vin = (const S*)w.v[d];
    S* uo = (S*)w.u[d];
    const int grid = lv.nbox * ntile;
    const double kup = d > 0 ? (double)lv.ksum : 0.0;
    prof_begin(P_UP, st);
    if (smem <= stage_limit) {
      RS_CUDA(cudaFuncSetAttribute(k_up<S, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_limit));
      RS_CUDA(cudaFuncSetAttribute(k_up<S, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_limit));
      if (CT == 1) k_up<S, 1, true><<<grid, SV_NT, smem, st>>>(bv, lv.uoff, U, vin, uo, cout, R, ntile);
      else k_up<S, 32, true><<<grid, SV_NT, smem, st>>>(bv, lv.uoff, U, vin, uo, cout, R, ntile);
    } else {
      if (CT == 1) k_up<S, 1, false><<<grid, SV_NT, 0, st>>>(bv, lv.uoff, U, vin, uo, cout, R, ntile);
      else k_up<S, 32, false><<<grid, SV_NT, 0, st>>>(bv, lv.uoff, U, vin, uo, cout, R, ntile);
    }
    RS_CHECK_LAUNCH();
    prof_end(P_UP, st, sS * ((double)lv.usz + (double)R * (2.0 * lv.ntot + kup)), 2.0 * cf * lv.usz * R);
  }
  for (int d = 1; d <= L; ++d) {
    const Level& lv = h->lv[d];
    const S* Lf = (const S*)(prec == RS_PREC_FP64 ? lv.Lf : lv.Lf32);
    size_t smem = sizeof(S) * (size_t)std::max(1, lv.maxk) * CT;
    const S* xp = (const S*)w.u[d - 1];
    S* uo = (S*)w.u[d];
    const int grid = lv.nbox * ntile;
    BoxView bv = box_view(lv);
    prof_begin(P_DOWN, st);
    if (smem <= stage_limit) {
      RS_CUDA(cudaFuncSetAttribute(k_down<S, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_limit));
      RS_CUDA(cudaFuncSetAttribute(k_down<S, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_limit));
      if (CT == 1) k_down<S, 1, true><<<grid, SV_NT, smem, st>>>(bv, lv.loff, Lf, xp, uo, R, ntile);
      else k_down<S, 32, true><<<grid, SV_NT, smem, st>>>(bv, lv.loff, Lf, xp, uo, R, ntile);
    } else {
      if (CT == 1) k_down<S, 1, false><<<grid, SV_NT, 0, st>>>(bv, lv.loff, Lf, xp, uo, R, ntile);
      else k_down<S, 32, false><<<grid, SV_NT, 0, st>>>(bv, lv.loff, Lf, xp, uo, R, ntile);
    }
    RS_CHECK_LAUNCH();
    prof_end(P_DOWN, st, sS * ((double)lv.lsz + (double)R * (2.0 * lv.ntot + lv.ksum)), 2.0 * cf * lv.lsz * R);
  }
  prof_begin(P_PERM, st);
  k_perm_out<S, SIO><<<nb, 256, 0, st>>>((const S*)w.u[L], h->perm, N, R, X, ldx);
  RS_CHECK_LAUNCH();
  prof_end(P_PERM, st, (double)N * R * (sS + sIO) + 4.0 * N, 0.0);
  return RS_OK;
}

int ensure_fwd(Handle* h, int R, cudaStream_t st) {
  if (h->fR >= R) return RS_OK;
  for (void* p : h->fz) if (p) RS_CUDA(cudaFreeAsync(p, st));
  for (void* p : h->fy) if (p) RS_CUDA(cudaFreeAsync(p, st));
  h->fz.assign(h->L + 1, nullptr);
  h->fy.assign(h->L + 1, nullptr);
  size_t sb = h->cplx ? sizeof(c128) : sizeof(double);
  for (int d = 0; d <= h->L; ++d) {
    size_t cnt = (size_t)std::max<int64_t>(1, h->lv[d].ntot) * R;
    RS_CUDA(cudaMallocAsync(&h->fz[d], cnt * sb, st));
    RS_CUDA(cudaMallocAsync(&h->fy[d], cnt * sb, st));
  }
  h->fR = R;
  return RS_OK;
}

FwdView fwd_view(const Handle* h, int d) {
  const Level& lv = h->lv[d];
  return FwdView{lv.n, lv.k, lv.off, lv.skoff, lv.act, lv.owner, lv.lperm, lv.toff, d == h->L,
                 lv.act_r ? lv.act_r : lv.act, lv.lperm_r ? lv.lperm_r : lv.lperm};
}

// y (tree order, point-major, in h->fy[L]) = A_RS z, z given in h->fz[L].
template <class S>
int forward_tree(Handle* h, int R, cudaStream_t st) {
  const int L = h->L;
  Pts pts;
  pts.x = h->pts;
  pts.y = h->pts + h->N;
  pts.z = h->dim == 3 ? h->pts + 2 * h->N : nullptr;
  pts.nx = h->dlg;
  pts.ny = h->dlg ? h->dlg + h->N : nullptr;
  pts.kap = h->dlg ? h->dlg + 2 * h->N : nullptr;
  const int nct = div_up(R, FD_CT);
  for (int d = L; d >= 0; --d) {
    const Level& lv = h->lv[d];
    FwdView fv = fwd_view(h, d);
    const double sS = sizeof(S), cf = is_cplx<S>::value ? 4.0 : 1.0;
    if (d > 0) {
      prof_begin(P_FWD_PROJ, st);
      k_fwd_proj<S><<<lv.nbox, 128, 0, st>>>(fv, (const S*)lv.T, (const S*)h->fz[d], (S*)h->fz[d - 1], R);
      RS_CHECK_LAUNCH();
      double tk = 0.0;
      for (int b = 0; b < lv.nbox; ++b) tk += (double)lv.h_k[b] * (lv.h_n[b] - lv.h_k[b]);
      prof_end(P_FWD_PROJ, st, sS * (tk + (double)R * (lv.ntot + lv.ksum)), 2.0 * cf * tk * R);
    }
    const int nrt = div_up(std::max(1, lv.maxn), FD_RT);
    double n2 = 0.0;
    for (int b = 0; b < lv.nbox; ++b) n2 += (double)lv.h_n[b] * lv.h_n[b];
    prof_begin(P_FWD_DBLOCK, st);
    k_fwd_dblock<S><<<lv.nbox * nrt * nct, SV_NT, 0, st>>>(fv, h->kp, pts, (const S*)h->fz[d], (S*)h->fy[d], R,
                                                           nrt, nct);
    RS_CHECK_LAUNCH();
    prof_end(P_FWD_DBLOCK, st, sS * 2.0 * R * lv.ntot, 2.0 * cf * n2 * R);
  }
  for (int d = 1; d <= L; ++d) {
    const Level& lv = h->lv[d];
    prof_begin(P_FWD_DOWN, st);
    k_fwd_down<S><<<lv.nbox, 128, 0, st>>>(fwd_view(h, d), (const S*)(lv.T_r ? lv.T_r : lv.T), (const S*)h->fy[d - 1],
                                           (S*)h->fy[d], R);
    RS_CHECK_LAUNCH();
    prof_end(P_FWD_DOWN, st, 0.0, 0.0);
  }
  return RS_OK;
}

template <class S>
int matvec_impl(Handle* h, const S* X, int64_t ldx, int R, S* Y, int64_t ldy, cudaStream_t st) {
  RS_TRY(ensure_fwd(h, R, st));
  int nb = div_up(h->N * R, 256);
  k_perm_in<S, S><<<nb, 256, 0, st>>>(X, ldx, h->perm, h->N, R, (S*)h->fz[h->L]);
  RS_CHECK_LAUNCH();
  RS_TRY(forward_tree<S>(h, R, st));
  k_perm_out<S, S><<<nb, 256, 0, st>>>((const S*)h->fy[h->L], h->perm, h->N, R, Y, ldy);
  RS_CHECK_LAUNCH();
  return RS_OK;
}



}  // namespace

int ensure_work_pub(Handle* h, int prec, int R, cudaStream_t st) { return ensure_work(h, prec, R, st); }

int solve_device(Handle* h, int prec, const void* d_B, int64_t ldb, int nrhs, void* d_X, int64_t ldx,
                 cudaStream_t st) {
  if (h->cplx) {
    if (prec == RS_PREC_FP64)
      return solve_impl<c128, c128>(h, prec, (const c128*)d_B, ldb, nrhs, (c128*)d_X, ldx, st);
    return solve_impl<c64, c128>(h, prec, (const c128*)d_B, ldb, nrhs, (c128*)d_X, ldx, st);
  }
  if (prec == RS_PREC_FP64)
    return solve_impl<double, double>(h, prec, (const double*)d_B, ldb, nrhs, (double*)d_X, ldx, st);
  return solve_impl<float, double>(h, prec, (const double*)d_B, ldb, nrhs, (double*)d_X, ldx, st);
}

int matvec_device(Handle* h, const void* d_X, int64_t ldx, int nrhs, void* d_Y, int64_t ldy, cudaStream_t st) {
  if (h->cplx) return matvec_impl<c128>(h, (const c128*)d_X, ldx, nrhs, (c128*)d_Y, ldy, st);
  return matvec_impl<double>(h, (const double*)d_X, ldx, nrhs, (double*)d_Y, ldy, st);
}

int colnorm2_device(Handle* h, const void* d_v, int nrhs, double* d_out, cudaStream_t st) {
  if (h->cplx) k_colnorm2<c128><<<nrhs, SV_NT, 0, st>>>((const c128*)d_v, h->N, d_out);
  else k_colnorm2<double><<<nrhs, SV_NT, 0, st>>>((const double*)d_v, h->N, d_out);
  RS_CHECK_LAUNCH();
  return RS_OK;
}

int axpy_lowp_device(Handle* h, void* d_x, const void* d_d, int nrhs, cudaStream_t st) {
  int64_t cnt = h->N * nrhs;
  if (h->cplx) k_axpy<c128><<<div_up(cnt, 256), 256, 0, st>>>((c128*)d_x, (const c128*)d_d, cnt);
  else k_axpy<double><<<div_up(cnt, 256), 256, 0, st>>>((double*)d_x, (const double*)d_d, cnt);
  RS_CHECK_LAUNCH();
  return RS_OK;
}

}  // namespace rs

// ----------------------------------------------------- allocation-free solve
// rs_solve_noalloc: the same level-by-level solve as rs_solve, for callers
// that must not allocate device memory during a solve -- for example a
// latency-critical serving loop, where cudaMalloc/cudaFree can synchronize
// the whole device and stall other streams, or a process that fixed its
// device-memory budget at start-up.  Its per-level vectors live in one
// file-scope device array of RS_NOALLOC_SCRATCH_BYTES that every GPU which
// loads the library holds until the process exits.
namespace rs {

static __device__ __align__(256) unsigned char g_noalloc_scratch[RS_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device (host code may
// not use the symbol itself).  Looked up once per device, on its first call.
int noalloc_scratch(void** out) {
  int dev = 0;
  RS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(RS_ERR_ARG, "rs_solve_noalloc: device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fail(RS_ERR_CUDA, "rs_solve_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return RS_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <class S, class SIO>
int solve_noalloc_impl(Handle* h, int prec, const SIO* B, int64_t ldb, int R, SIO* X, int64_t ldx,
                       cudaStream_t st) {
  const int64_t N = h->N;
  const int L = h->L;
  size_t need = 0;
  for (int d = 0; d <= L; ++d) need += 2 * align256(sizeof(S) * (size_t)std::max<int64_t>(1, h->lv[d].ntot) * R);
  if (need > (size_t)RS_NOALLOC_SCRATCH_BYTES)
    return fail(RS_ERR_ARG, "rs_solve_noalloc: needs %zu bytes of scratch for nrhs=%d, limit %zu; use fewer columns",
                need, R, (size_t)RS_NOALLOC_SCRATCH_BYTES);
  void* base = nullptr;
  RS_TRY(noalloc_scratch(&base));
  std::vector<S*> v(L + 1), u(L + 1);
  unsigned char* p = (unsigned char*)base;
  for (int d = 0; d <= L; ++d) {
    size_t b = align256(sizeof(S) * (size_t)std::max<int64_t>(1, h->lv[d].ntot) * R);
    v[d] = (S*)p;
    p += b;
    u[d] = (S*)p;
    p += b;
  }
  int nb = div_up(N * R, 256);
  k_perm_in<SIO, S><<<nb, 256, 0, st>>>(B, ldb, h->perm, N, R, v[L]);
  RS_CHECK_LAUNCH();
  const int CT = R == 1 ? 1 : 32;
  const int ntile = div_up(R, CT);
  const size_t stage_limit = 96 * 1024;
  for (int d = L; d >= 0; --d) {
    const Level& lv = h->lv[d];
    const S* U = (const S*)(prec == RS_PREC_FP64 ? lv.U : lv.U32);
    S* cout = d > 0 ? v[d - 1] : nullptr;
    size_t smem = sizeof(S) * (size_t)std::max(1, lv.maxn) * CT;
    BoxView bv = box_view(lv);
    if (d == 0) bv.skoff = nullptr;
    const int grid = lv.nbox * ntile;
    if (smem <= stage_limit) {
      RS_CUDA(cudaFuncSetAttribute(k_up<S, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_limit));
      RS_CUDA(cudaFuncSetAttribute(k_up<S, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_limit));
      if (CT == 1) k_up<S, 1, true><<<grid, SV_NT, smem, st>>>(bv, lv.uoff, U, v[d], u[d], cout, R, ntile);
      else k_up<S, 32, true><<<grid, SV_NT, smem, st>>>(bv, lv.uoff, U, v[d], u[d], cout, R, ntile);
    } else {
      if (CT == 1) k_up<S, 1, false><<<grid, SV_NT, 0, st>>>(bv, lv.uoff, U, v[d], u[d], cout, R, ntile);
      else k_up<S, 32, false><<<grid, SV_NT, 0, st>>>(bv, lv.uoff, U, v[d], u[d], cout, R, ntile);
    }
    RS_CHECK_LAUNCH();
  }
  for (int d = 1; d <= L; ++d) {
    const Level& lv = h->lv[d];
    const S* Lf = (const S*)(prec == RS_PREC_FP64 ? lv.Lf : lv.Lf32);
    size_t smem = sizeof(S) * (size_t)std::max(1, lv.maxk) * CT;
    const int grid = lv.nbox * ntile;
    BoxView bv = box_view(lv);
    if (smem <= stage_limit) {
      RS_CUDA(cudaFuncSetAttribute(k_down<S, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_limit));
      RS_CUDA(cudaFuncSetAttribute(k_down<S, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_limit));
      if (CT == 1) k_down<S, 1, true><<<grid, SV_NT, smem, st>>>(bv, lv.loff, Lf, u[d - 1], u[d], R, ntile);
      else k_down<S, 32, true><<<grid, SV_NT, smem, st>>>(bv, lv.loff, Lf, u[d - 1], u[d], R, ntile);
    } else {
      if (CT == 1) k_down<S, 1, false><<<grid, SV_NT, 0, st>>>(bv, lv.loff, Lf, u[d - 1], u[d], R, ntile);
      else k_down<S, 32, false><<<grid, SV_NT, 0, st>>>(bv, lv.loff, Lf, u[d - 1], u[d], R, ntile);
    }
    RS_CHECK_LAUNCH();
  }
  k_perm_out<S, SIO><<<nb, 256, 0, st>>>(u[L], h->perm, N, R, X, ldx);
  RS_CHECK_LAUNCH();
  return RS_OK;
}

}  // namespace

int solve_noalloc_device(Handle* h, int prec, const void* d_B, int64_t ldb, int nrhs, void* d_X, int64_t ldx,
                         cudaStream_t st) {
  if (h->cplx) {
    if (prec == RS_PREC_FP64)
      return solve_noalloc_impl<c128, c128>(h, prec, (const c128*)d_B, ldb, nrhs, (c128*)d_X, ldx, st);
    return solve_noalloc_impl<c64, c128>(h, prec, (const c128*)d_B, ldb, nrhs, (c128*)d_X, ldx, st);
  }
  if (prec == RS_PREC_FP64)
    return solve_noalloc_impl<double, double>(h, prec, (const double*)d_B, ldb, nrhs, (double*)d_X, ldx, st);
  return solve_noalloc_impl<float, double>(h, prec, (const double*)d_B, ldb, nrhs, (double*)d_X, ldx, st);
}

}  // namespace rs
