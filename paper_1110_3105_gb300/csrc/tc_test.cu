// Self-test of the tensor-core building blocks (tc.cuh): one 128 x N x K
// block product D = A B^T through shared-memory descriptors and tensor
// memory, for checking the operand layout and descriptors against a host
// product.  Not part of the solver's path.
#include <cuda_bf16.h>

#include "rs_internal.h"
#include "tc.cuh"

namespace rs {
namespace {

constexpr int ST_NT = 128;

// A: 128 x K row-major fp32, B: N x K row-major fp32 (K = 32 for tf32, 64 for
// bf16: one 128-byte row); D: 128 x N row-major fp32.  kind 0 = tf32 (the
// fp32 values are rounded to tf32), 1 = bf16 (rounded to bf16).
template <int KIND>
__global__ void __launch_bounds__(ST_NT) k_tc_selftest(const float* A, const float* B, float* D, int N,
                                                       int* status) {
  extern __shared__ unsigned char st_raw[];
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) uint64_t s_bar;
  constexpr int ES = KIND == 0 ? 4 : 2, K = 128 / ES;
  // 1024-byte aligned operand area
  const uint32_t raw = tc::smem_u32(st_raw);
  unsigned char* base = st_raw + ((1024u - (raw & 1023u)) & 1023u);
  unsigned char* As = base;
  unsigned char* Bs = base + 128 * 128;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint32_t ncols = 32;
  while ((int)ncols < N) ncols <<= 1;
  if (warp == 0) tc::tmem_alloc(&s_taddr, ncols);
  if (tid == 0) tc::mbar_init(&s_bar, 1);
  for (int e = tid; e < 128 * K; e += ST_NT) {
    const int r = e / K, k = e % K;
    const float v = A[e];
    if (KIND == 0) *reinterpret_cast<float*>(As + tc::sw128_offset(r, k, 4)) = tc::tf32_hi(v);
    else *reinterpret_cast<__nv_bfloat16*>(As + tc::sw128_offset(r, k, 2)) = __float2bfloat16_rn(v);
  }
  for (int e = tid; e < N * K; e += ST_NT) {
    const int r = e / K, k = e % K;
    const float v = B[e];
    if (KIND == 0) *reinterpret_cast<float*>(Bs + tc::sw128_offset(r, k, 4)) = tc::tf32_hi(v);
    else *reinterpret_cast<__nv_bfloat16*>(Bs + tc::sw128_offset(r, k, 2)) = __float2bfloat16_rn(v);
  }
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = s_taddr;
  if (tid == 0) {
    const uint32_t id = tc::idesc(KIND == 0 ? tc::FMT_TF32 : tc::FMT_BF16, 128, N);
    for (int ks = 0; ks < 4; ++ks) {
      const uint64_t ad = tc::desc_sw128(tc::smem_u32(As) + 32 * ks);
      const uint64_t bd = tc::desc_sw128(tc::smem_u32(Bs) + 32 * ks);
      if (KIND == 0) tc::mma_tf32(taddr, ad, bd, id, ks > 0);
      else tc::mma_f16(taddr, ad, bd, id, ks > 0);
    }
    tc::mma_commit(&s_bar);
  }
  __syncwarp();
  const bool ok = tc::mbar_wait(&s_bar, 0, 1 << 22);
  if (!ok && lane == 0) atomicExch(status, 1);
  tc::fence_after_sync();
  if (ok) {
    const int row = 32 * (warp & 3) + lane;
    for (int c = 0; c < N; c += 16) {
      float v[16];
      tc::tmem_ld16(taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c, v);
      tc::tmem_ld_wait();
      for (int i = 0; i < 16; ++i) D[(size_t)row * N + c + i] = v[i];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(taddr, ncols);
}

}  // namespace
}  // namespace rs

extern "C" int rs_tc_selftest(int kind, const float* A, const float* B, float* D, int n) {
  using namespace rs;
  if ((kind != 0 && kind != 1) || !A || !B || !D || n < 16 || n > 256 || n % 16)
    return fail(RS_ERR_ARG, "rs_tc_selftest: bad arguments");
  int* st = nullptr;
  RS_CUDA(cudaMalloc((void**)&st, sizeof(int)));
  RS_CUDA(cudaMemset(st, 0, sizeof(int)));
  const size_t smem = 1024 + 128 * 128 + (size_t)n * 128;
  int rc = RS_OK;
  if (kind == 0) {
    RS_CUDA(cudaFuncSetAttribute(k_tc_selftest<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_tc_selftest<0><<<1, ST_NT, smem>>>(A, B, D, n, st);
  } else {
    RS_CUDA(cudaFuncSetAttribute(k_tc_selftest<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_tc_selftest<1><<<1, ST_NT, smem>>>(A, B, D, n, st);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int hs = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&hs, st, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(st);
  if (e != cudaSuccess) rc = fail(RS_ERR_CUDA, "rs_tc_selftest: %s", cudaGetErrorString(e));
  else if (hs) rc = fail(RS_ERR_TIMEOUT, "rs_tc_selftest: MMA completion wait ran out");
  return rc;
}
