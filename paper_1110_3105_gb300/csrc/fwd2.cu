// Double-float forward operator for the refinement residual (real kernels).
//
// The residual r = b - A_RS x of the refinement (forward operator of eq.
// multilevel-compression, applied as in Sec. 3.3) must be accurate to far
// below the 1e-10 target.  On GB300 FP64 FMAs run at 1/57 of the FP32 rate,
// so the products are formed in double-float arithmetic on the FP32 pipes:
// every value is an unevaluated sum hi + lo of two floats (about 48
// significant bits), products use the exact FMA-based two-product and sums
// the exact two-sum (Dekker 1971; Knuth, TAOCP vol. 2, Sec. 4.2.2), giving a
// relative error near 2^-46 per dot product.
//
// The kernel blocks D^(l) of the forward operator (leaf: A(I_i, I_i);
// above: w G between skeletons of different children, zero within one
// child; root: the same form) are evaluated once per build in FP64 from the
// coordinates and stored as (hi, lo) pairs, as is T.
//
// A second mode (F32) runs the same kernels with float arithmetic on the hi
// parts only; it serves the cheap update r_{j+1} = r_j - A d_j of the
// refinement, whose correction d_j is already ~1e-7 of x.
#include <algorithm>
#include <vector>

#include "rs_internal.h"

namespace rs {

namespace {

struct df {
  float hi, lo;
};

// Explicitly rounded operations throughout: the compiler must not fuse a
// product into a following sum, or the two-product / two-sum lose exactness.
__device__ __forceinline__ df df_split(double x) {
  float h = __double2float_rn(x);
  return df{h, __double2float_rn(__dsub_rn(x, (double)h))};
}

// s += a * b (double-float), a, b exact float pairs.
__device__ __forceinline__ void df_mac(df& s, df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);           // exact error of the product
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float t = __fadd_rn(s.hi, p);                  // two-sum of s.hi and p
  float bb = __fsub_rn(t, s.hi);
  float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  s.lo = __fadd_rn(s.lo, __fadd_rn(err, e));
  s.hi = t;
}
__device__ __forceinline__ void df_add(df& s, df b) {
  float t = __fadd_rn(s.hi, b.hi);
  float bb = __fsub_rn(t, s.hi);
  float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bb)), __fsub_rn(b.hi, bb));
  s.lo = __fadd_rn(s.lo, __fadd_rn(err, b.lo));
  s.hi = t;
}
__device__ __forceinline__ df df_norm(df s) {
  float t = __fadd_rn(s.hi, s.lo);
  return df{t, __fsub_rn(s.lo, __fsub_rn(t, s.hi))};
}

template <bool DF>
__device__ __forceinline__ void mac(df& s, df a, df b) {
  if (DF) df_mac(s, a, b);
  else s.hi = fmaf(a.hi, b.hi, s.hi);
}
template <bool DF>
__device__ __forceinline__ void add(df& s, df b) {
  if (DF) df_add(s, b);
  else s.hi += b.hi;
}

constexpr int F_NT = 256;

struct FwdTab {
  const int* n;
  const int* k;
  const int64_t* off;
  const int64_t* skoff;
  const int* lperm;
  const int64_t* toff;
  const int64_t* dfoff;
};

// Kernel blocks of one depth in FP64, stored as (hi, lo) pairs.
__global__ void k_dfw_fill(FwdTab t, KParams kp, Pts pts, const int* act, const int* owner, int leaf_level,
                           df* D) {
  const int b = blockIdx.x;
  const int n = t.n[b];
  const int64_t off = t.off[b];
  df* Db = D + t.dfoff[b];
  for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
    int r = (int)(e % n), c = (int)(e / n);
    double v;
    if (leaf_level) v = system_entry<double>(kp, pts, act[off + r], act[off + c]);
    else v = owner[off + r] == owner[off + c] ? 0.0 : offdiag_entry<double>(kp, pts, act[off + r], act[off + c]);
    Db[e] = df_split(v);
  }
}

__global__ void k_df_from_double(const double* in, df* out, int64_t cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) out[i] = df_split(in[i]);
}

// z[pos*R + c] = split(x[perm[pos] + c*ldx])
template <bool DF>
__global__ void k_df_in(const double* x, int64_t ldx, const int* perm, int64_t N, int R, df* z) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * R) return;
  int64_t i = e / R;
  int c = (int)(e % R);
  double v = x[perm[i] + (int64_t)c * ldx];
  z[e] = DF ? df_split(v) : df{(float)v, 0.0f};
}

// r[perm[i] + c*N] = b[...] - y   (FP64 result)
__global__ void k_df_res(const double* b, const df* y, const int* perm, int64_t N, int R, double* r) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * R) return;
  int64_t i = e / R;
  int c = (int)(e % R);
  int64_t g = perm[i] + (int64_t)c * N;
  df v = y[e];
  r[g] = (b[g] - (double)v.hi) - (double)v.lo;
}

// Shared routine for one box and one column tile.  The CTA's 8 warps form
// a WR x WC grid: warp (wr, wc) owns output rows o0 + 32 wr + lane (lanes own
// rows, so the factor loads A(o, q) = A[o * sa_o + q * sa_q] of a warp are
// contiguous when sa_o = 1) and columns c0 + CT wc + [0, CT) in registers.
// B rows (gathered through brow) are staged QC at a time in shared memory;
// emit(o, c, value) stores each result.
constexpr int F_QC = 64;
template <bool DF, int CT, int WC, class BRow, class Emit>
__device__ void tile_gemm(const df* A, int64_t sa_o, int64_t sa_q, int nout, int K, const df* Bv, BRow brow, int R,
                          int c0, df* sB, Emit emit) {
  constexpr int WR = (F_NT / 32) / WC;
  constexpr int TC = CT * WC;   // columns of the CTA tile
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wr = warp / WC, wc = warp % WC;
  const int cbase = wc * CT;
  // row chunks of 32 WR rows are spread over the grid (blockIdx.y)
  for (int o0 = blockIdx.y * 32 * WR; o0 < nout; o0 += gridDim.y * 32 * WR) {
    const int o = o0 + wr * 32 + lane;
    df acc[CT];
#pragma unroll
    for (int c = 0; c < CT; ++c) acc[c] = df{0.0f, 0.0f};
    for (int q0 = 0; q0 < K; q0 += F_QC) {
      const int qn = min(F_QC, K - q0);
      __syncthreads();
      for (int e = threadIdx.x; e < qn * TC; e += F_NT) {
        int q = e / TC, c = e % TC;
        sB[e] = c0 + c < R ? Bv[brow(q0 + q) * R + c0 + c] : df{0.0f, 0.0f};
      }
      __syncthreads();
      if (o < nout) {
        const df* Ar = A + (int64_t)o * sa_o + (int64_t)q0 * sa_q;
        for (int qq = 0; qq < qn; qq += 8) {
          df a[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) a[j] = qq + j < qn ? Ar[(int64_t)(qq + j) * sa_q] : df{0.0f, 0.0f};
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            if (qq + j < qn) {
#pragma unroll
              for (int c = 0; c < CT; ++c) mac<DF>(acc[c], a[j], sB[(qq + j) * TC + cbase + c]);
            }
          }
        }
      }
    }
    if (o < nout) {
#pragma unroll
      for (int c = 0; c < CT; ++c)
        if (c0 + cbase + c < R) emit(o, cbase + c, acc[c]);
    }
  }
}

// Largest box the staged tile supports (rows of B in shared memory).
constexpr int F_MAXK = 320;

// y_d (per box rows) = D z_d
template <bool DF, int CT, int WC>
__global__ void __launch_bounds__(F_NT) k_df_dblock(FwdTab t, const df* D, const df* z, df* y, int R, int ntile) {
  extern __shared__ __align__(16) unsigned char smem[];
  df* sB = reinterpret_cast<df*>(smem);
  const int b = blockIdx.x / ntile, c0 = (blockIdx.x % ntile) * CT * WC;
  const int n = t.n[b];
  const int64_t off = t.off[b];
  tile_gemm<DF, CT, WC>(D + t.dfoff[b], 1, n, n, n, z, [=](int q) { return off + q; }, R, c0, sB,
                    [=](int o, int c, df s) { y[(off + o) * R + c0 + c] = df_norm(s); });
}

// z_parent[skoff + a] = z[sk_a] + sum_e T[a, e] z[rd_e]
template <bool DF, int CT, int WC>
__global__ void __launch_bounds__(F_NT) k_df_proj(FwdTab t, const df* T, const df* z, df* zpar, int R, int ntile) {
  extern __shared__ __align__(16) unsigned char smem[];
  df* sB = reinterpret_cast<df*>(smem);
  const int b = blockIdx.x / ntile, c0 = (blockIdx.x % ntile) * CT * WC;
  const int n = t.n[b], k = t.k[b];
  const int64_t off = t.off[b], sk = t.skoff[b];
  const int* lp = t.lperm + off;
  tile_gemm<DF, CT, WC>(T + t.toff[b], 1, k, k, n - k, z, [=](int q) { return off + lp[k + q]; }, R, c0, sB,
                    [=](int a, int c, df s) {
                      add<DF>(s, z[(off + lp[a]) * R + c0 + c]);
                      zpar[(sk + a) * R + c0 + c] = df_norm(s);
                    });
}

// y[sk_a] += w[a];  y[rd_e] += sum_a T[a, e] w[a]   (w = y_parent[skoff ...])
template <bool DF, int CT, int WC>
__global__ void __launch_bounds__(F_NT) k_df_down(FwdTab t, const df* T, const df* ypar, df* y, int R, int ntile) {
  extern __shared__ __align__(16) unsigned char smem[];
  df* sB = reinterpret_cast<df*>(smem);
  const int b = blockIdx.x / ntile, c0 = (blockIdx.x % ntile) * CT * WC, cw = min(CT * WC, R - c0);
  const int n = t.n[b], k = t.k[b], nr = n - k;
  const int64_t off = t.off[b], sk = t.skoff[b];
  const int* lp = t.lperm + off;
  // rows e of T^T (nr x k): T^T(e, a) = T[a + e k]
  tile_gemm<DF, CT, WC>(T + t.toff[b], k, 1, nr, k, ypar, [=](int q) { return sk + q; }, R, c0, sB,
                    [=](int e, int c, df s) {
                      int64_t idx = (off + lp[k + e]) * R + c0 + c;
                      df v = y[idx];
                      add<DF>(v, s);
                      y[idx] = df_norm(v);
                    });
  if (blockIdx.y == 0)   // skeleton rows once per box (the grid's row chunks cover the redundant rows)
  for (int e = threadIdx.x; e < k * cw; e += F_NT) {
    int a = e / cw, c = e % cw;
    int64_t idx = (off + lp[a]) * R + c0 + c;
    df v = y[idx];
    add<DF>(v, ypar[(sk + a) * R + c0 + c]);
    y[idx] = df_norm(v);
  }
}

FwdTab fwd_tab(const Level& lv) { return FwdTab{lv.n, lv.k, lv.off, lv.skoff, lv.lperm, lv.toff, lv.dfoff}; }

template <bool DF, int CT, int WC>
int set_df_smem_ct() {
  const int lim = (int)(sizeof(df) * CT * WC * F_QC);
  if (lim <= 48 * 1024) return RS_OK;   // default limit suffices for this shape
  RS_CUDA(cudaFuncSetAttribute(k_df_dblock<DF, CT, WC>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  RS_CUDA(cudaFuncSetAttribute(k_df_proj<DF, CT, WC>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  RS_CUDA(cudaFuncSetAttribute(k_df_down<DF, CT, WC>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  return RS_OK;
}

int set_df_smem() {
  static bool done = false;
  if (done) return RS_OK;
  RS_TRY((set_df_smem_ct<true, 1, 1>()));
  RS_TRY((set_df_smem_ct<true, 2, 8>()));
  RS_TRY((set_df_smem_ct<true, 16, 8>()));
  RS_TRY((set_df_smem_ct<false, 1, 1>()));
  RS_TRY((set_df_smem_ct<false, 2, 8>()));
  RS_TRY((set_df_smem_ct<false, 16, 8>()));
  done = true;
  return RS_OK;
}

int ensure_df(Handle* h, int R, cudaStream_t st) {
  RS_TRY(set_df_smem());
  if (h->dfR >= R) return RS_OK;
  for (void* p : h->dfz) if (p) RS_CUDA(cudaFreeAsync(p, st));
  for (void* p : h->dfy) if (p) RS_CUDA(cudaFreeAsync(p, st));
  h->dfz.assign(h->L + 1, nullptr);
  h->dfy.assign(h->L + 1, nullptr);
  for (int d = 0; d <= h->L; ++d) {
    size_t cnt = (size_t)std::max<int64_t>(1, h->lv[d].ntot) * R;
    RS_CUDA(cudaMallocAsync(&h->dfz[d], cnt * sizeof(df), st));
    RS_CUDA(cudaMallocAsync(&h->dfy[d], cnt * sizeof(df), st));
  }
  h->dfR = R;
  return RS_OK;
}

// Row chunks of a level's largest box (32 rows per warp row of the CTA).
int rchunks(int maxrows, int WC) {
  const int WR = (F_NT / 32) / WC;
  return std::max(1, div_up(std::max(1, maxrows), 32 * WR));
}

template <bool DF, int CT, int WC>
int forward_df_ct(Handle* h, const double* x, int64_t ldx, int R, cudaStream_t st) {
  RS_TRY(ensure_df(h, R, st));
  const int L = h->L;
  const int ntile = div_up(R, CT * WC);
  const size_t smem = sizeof(df) * CT * WC * F_QC;
  int nb = div_up(h->N * R, 256);
  const int cat = DF ? P_RESID : P_MISC;
  prof_begin(cat, st);
  k_df_in<DF><<<nb, 256, 0, st>>>(x, ldx, h->perm, h->N, R, (df*)h->dfz[L]);
  RS_CHECK_LAUNCH();
  double macs = 0.0, bytes = 0.0;
  for (int d = L; d >= 0; --d) {
    const Level& lv = h->lv[d];
    if (lv.maxn > F_MAXK) return fail(RS_ERR_ARG, "refinement: box of %d points exceeds the tile limit", lv.maxn);
    if (d > 0) {
      k_df_proj<DF, CT, WC><<<dim3(lv.nbox * ntile, rchunks(lv.maxk, WC)), F_NT, smem, st>>>(fwd_tab(lv), (const df*)lv.Tdf, (const df*)h->dfz[d],
                                                             (df*)h->dfz[d - 1], R, ntile);
      RS_CHECK_LAUNCH();
    }
    k_df_dblock<DF, CT, WC><<<dim3(lv.nbox * ntile, rchunks(lv.maxn, WC)), F_NT, smem, st>>>(fwd_tab(lv), (const df*)lv.Dfw, (const df*)h->dfz[d],
                                                             (df*)h->dfy[d], R, ntile);
    RS_CHECK_LAUNCH();
    macs += (double)R * ((double)lv.dfsz + 2.0 * (double)lv.tsz_used);
    bytes += 8.0 * ((double)lv.dfsz + 2.0 * lv.tsz_used) + 8.0 * R * 4.0 * lv.ntot;
  }
  for (int d = 1; d <= L; ++d) {
    const Level& lv = h->lv[d];
    k_df_down<DF, CT, WC><<<dim3(lv.nbox * ntile, rchunks(lv.maxn, WC)), F_NT, smem, st>>>(fwd_tab(lv), (const df*)lv.Tdf, (const df*)h->dfy[d - 1],
                                                           (df*)h->dfy[d], R, ntile);
    RS_CHECK_LAUNCH();
  }
  prof_end(cat, st, bytes, 2.0 * macs);
  return RS_OK;
}

// Tile shape by batch width: one column (warps over rows), up to 16 columns
// (2 per warp), wider (16 per warp, 128 per CTA).
template <bool DF>
int forward_df(Handle* h, const double* x, int64_t ldx, int R, cudaStream_t st) {
  if (R == 1) return forward_df_ct<DF, 1, 1>(h, x, ldx, R, st);
  if (R <= 16) return forward_df_ct<DF, 2, 8>(h, x, ldx, R, st);
  return forward_df_ct<DF, 16, 8>(h, x, ldx, R, st);
}

}  // namespace

// Build-time: kernel blocks of every depth and T as (hi, lo) pairs (real kernels).
int make_fwd_blocks(Handle* h, cudaStream_t st) {
  if (h->cplx) return RS_OK;
  Pts pts;
  pts.x = h->pts;
  pts.y = h->pts + h->N;
  pts.z = h->dim == 3 ? h->pts + 2 * h->N : nullptr;
  for (int d = 0; d <= h->L; ++d) {
    Level& lv = h->lv[d];
    std::vector<int64_t> dfoff(lv.nbox);
    int64_t acc = 0, tused = 0;
    for (int b = 0; b < lv.nbox; ++b) {
      dfoff[b] = acc;
      acc += (int64_t)lv.h_n[b] * lv.h_n[b];
      if (d > 0) tused += (int64_t)lv.h_k[b] * (lv.h_n[b] - lv.h_k[b]);
    }
    lv.dfsz = acc;
    lv.tsz_used = tused;
    RS_TRY(dalloc_t(h, &lv.dfoff, std::max(1, lv.nbox)));
    RS_CUDA(cudaMemcpyAsync(lv.dfoff, dfoff.data(), sizeof(int64_t) * lv.nbox, cudaMemcpyHostToDevice, st));
    RS_TRY(dalloc(h, &lv.Dfw, sizeof(df) * std::max<int64_t>(1, acc)));
    k_dfw_fill<<<lv.nbox, 256, 0, st>>>(fwd_tab(lv), h->kp, pts, lv.act, lv.owner, d == h->L, (df*)lv.Dfw);
    RS_CHECK_LAUNCH();
    if (d > 0 && lv.tsz > 0) {
      RS_TRY(dalloc(h, &lv.Tdf, sizeof(df) * lv.tsz));
      k_df_from_double<<<div_up(lv.tsz, 256), 256, 0, st>>>((const double*)lv.T, (df*)lv.Tdf, lv.tsz);
      RS_CHECK_LAUNCH();
    }
  }
  return RS_OK;
}

// The double-float residual covers real kernels whose boxes fit the staged tile.
bool df_supported(const Handle* h) {
  if (h->cplx) return false;
  for (const Level& lv : h->lv)
    if (lv.maxn > F_MAXK) return false;
  return true;
}

// r = b - A_RS x  (double-float products), or in place r -= A_RS d (float products).
int residual_df(Handle* h, const double* b, const double* x, double* r, int R, bool full, cudaStream_t st) {
  if (full) RS_TRY(forward_df<true>(h, x, h->N, R, st));
  else RS_TRY(forward_df<false>(h, x, h->N, R, st));
  int nb = div_up(h->N * R, 256);
  k_df_res<<<nb, 256, 0, st>>>(b, (const df*)h->dfy[h->L], h->perm, h->N, R, r);
  RS_CHECK_LAUNCH();
  return RS_OK;
}

}  // namespace rs
