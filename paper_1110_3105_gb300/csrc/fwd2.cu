// Forward operator for the refinement residual.
//
// The residual r = b - A_RS x of the refinement (forward operator of eq.
// multilevel-compression, applied as in Sec. 3.3) must be accurate to far
// below the 1e-10 target.  On GB300 FP64 FMAs run at 1/57 of the FP32 rate,
// so the products are formed in double-float arithmetic on the FP32 pipes:
// every value is an unevaluated sum hi + lo of two floats (about 48
// significant bits), products use the exact FMA-based two-product and sums
// the exact two-sum (Dekker 1971; Knuth, TAOCP vol. 2, Sec. 4.2.2).
//
// The forward operator has the same two-pass structure as the inverse
// (eq. multilevel-compression read right to left): upward, each box maps its
// input z to [D z ; P z] (the second part is its skeleton rows of the parent's
// input); the root applies its own kernel block; downward, each box adds
// P^T y_parent to its D z.  So it runs on the persistent solve kernel, with
// the factors FU = [D ; P] and FL = P^T built here once per build from the
// coordinates (FP64 evaluation) and stored as float and double-float.
//
// The float mode serves the cheap update r_{j+1} = r_j - A d_j of the
// refinement, whose correction d_j is already ~1e-7 of x.  Complex kernels
// store the same factors as complex float and complex double-float (each
// part a double-float), on the same persistent kernel.
#include <algorithm>
#include <vector>

#include "rs_internal.h"

namespace rs {

namespace {

struct FwdTab {
  const int* n;
  const int* k;
  const int64_t* off;
  const int64_t* skoff;
  const int* lperm;
  const int64_t* toff;
};

// Forward operator factors of one depth, in the solve's two-pass form:
//   FU = [D ; P] ((n+k) x n): rows 0..n-1, the kernel block D of the box, are
//        written by the factorization while it assembles its block (skel.cu:
//        emit_fwd); rows n.. hold the projection P = [I T] Pi;
//   FL = P^T (n x k).
// Stored as float and as double-float (real), complex float and complex
// double-float (complex).
template <class S> __device__ __forceinline__ void put_lo(void* p, int64_t i, S v);
template <> __device__ __forceinline__ void put_lo<double>(void* p, int64_t i, double v) {
  static_cast<float*>(p)[i] = f64_to_f32_rn(v);
}
template <> __device__ __forceinline__ void put_lo<c128>(void* p, int64_t i, c128 v) {
  static_cast<c64*>(p)[i] = c64(f64_to_f32_rn(v.re), f64_to_f32_rn(v.im));
}
template <class S> __device__ __forceinline__ void put_hi(void* p, int64_t i, S v);
template <> __device__ __forceinline__ void put_hi<double>(void* p, int64_t i, double v) {
  static_cast<dfloat*>(p)[i] = f64_to_df(v);
}
template <> __device__ __forceinline__ void put_hi<c128>(void* p, int64_t i, c128 v) {
  static_cast<cdfloat*>(p)[i] = cdfloat(f64_to_df(v.re), f64_to_df(v.im));
}

// FU's projection rows from the column ID (R_i = P_i), FL from the row ID
// (L_i = Q_i^T; Q = P for symmetric kernels).
template <class S>
__global__ void k_fwd_factors(FwdTab t, const S* T, const int* lperm_r, const S* Tr, const int64_t* uoff,
                              const int64_t* loff, void* FUlo, void* FUhi, void* FLlo, void* FLhi) {
  extern __shared__ int inv[];   // position within I -> index in the ID order (column ID, then row ID)
  const int b = blockIdx.x;
  const int n = t.n[b], k = t.k ? t.k[b] : 0, rows = n + k;
  if (k == 0) return;
  const int64_t off = t.off[b];
  const int* lp = t.lperm + off;
  const int* lpr = lperm_r + off;
  const S* Tb = T + t.toff[b];
  const S* Tbr = Tr + t.toff[b];
  int* invr = inv + n;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    inv[lp[q]] = q;
    invr[lpr[q]] = q;
  }
  __syncthreads();
  auto pval = [&](int a, int c) -> S {   // P[a, c]
    int q = inv[c];
    return q < k ? S(q == a ? 1.0 : 0.0) : Tb[a + (size_t)(q - k) * k];
  };
  auto qval = [&](int a, int c) -> S {   // Q[a, c]
    int q = invr[c];
    return q < k ? S(q == a ? 1.0 : 0.0) : Tbr[a + (size_t)(q - k) * k];
  };
  const int64_t ub = uoff[b], lb = loff[b];
  for (int64_t e = threadIdx.x; e < (int64_t)k * n; e += blockDim.x) {
    const int a = (int)(e % k), c = (int)(e / k);
    const S v = pval(a, c);
    const int64_t i = ub + n + a + (int64_t)c * rows;
    put_lo<S>(FUlo, i, v);
    put_hi<S>(FUhi, i, v);
  }
  for (int64_t e = threadIdx.x; e < (int64_t)n * k; e += blockDim.x) {
    const int r = (int)(e % n), a = (int)(e / n);
    const S v = qval(a, r);
    put_lo<S>(FLlo, lb + e, v);
    put_hi<S>(FLhi, lb + e, v);
  }
}

}  // namespace

// Build-time: the projection rows of the forward factors of every depth
// (the factors were allocated with the level's pools).
template <class S>
int fwd_blocks(Handle* h, cudaStream_t st) {
  for (int d = 1; d <= h->L; ++d) {
    Level& lv = h->lv[d];
    FwdTab t{lv.n, lv.k, lv.off, lv.skoff, lv.lperm, lv.toff};
    const size_t smem = 2 * sizeof(int) * (size_t)std::max(1, lv.maxn);
    RS_CUDA(cudaFuncSetAttribute(k_fwd_factors<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_fwd_factors<S><<<lv.nbox, 256, smem, st>>>(t, (const S*)lv.T, lv.lperm_r ? lv.lperm_r : lv.lperm,
                                                 (const S*)(lv.T_r ? lv.T_r : lv.T), lv.uoff, lv.loff, lv.FU32,
                                                 lv.FUdf, lv.FL32, lv.FLdf);
    RS_CHECK_LAUNCH();
  }
  return RS_OK;
}

int make_fwd_blocks(Handle* h, cudaStream_t st) {
  return h->cplx ? fwd_blocks<c128>(h, st) : fwd_blocks<double>(h, st);
}


// r = b - A_RS x with double-float products (full), or r = r - A_RS d with
// float products (update), complex variants for complex kernels (the buffers
// then hold complex double values): the forward operator runs on the
// persistent two-pass kernel with the forward factors, subtracting its
// result from b.
int residual_df(Handle* h, const double* b, const double* x, double* r, int R, bool full, cudaStream_t st) {
  return solve_pers_device_sub(h, full ? MODE_FWD_DF : MODE_FWD_F32, x, h->N, R, r, h->N, b, st);
}

}  // namespace rs
