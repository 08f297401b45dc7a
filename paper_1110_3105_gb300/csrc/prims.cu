// Device primitives used by the tree and the level bookkeeping:
// exclusive scans, a stable LSD radix sort of (key, value) pairs and small
// reductions.  All are deterministic (fixed reduction orders, stable ranks).
#include <algorithm>
#include <vector>

#include "rs_internal.h"

namespace rs {

namespace {

constexpr int SCAN_NT = 1024;
constexpr int SCAN_PER_BLOCK = 2 * SCAN_NT;

// Block-wide exclusive scan of SCAN_PER_BLOCK int64 values (two per thread).
template <class In>
__global__ void k_scan_blocks(const In* in, int64_t* out, int64_t n, int64_t* block_sums) {
  __shared__ int64_t s[SCAN_PER_BLOCK];
  int64_t base = (int64_t)blockIdx.x * SCAN_PER_BLOCK;
  int t = threadIdx.x;
  int64_t i0 = base + 2 * t, i1 = i0 + 1;
  s[2 * t] = i0 < n ? (int64_t)in[i0] : 0;
  s[2 * t + 1] = i1 < n ? (int64_t)in[i1] : 0;
  // up-sweep
  int offset = 1;
  for (int d = SCAN_PER_BLOCK >> 1; d > 0; d >>= 1) {
    __syncthreads();
    if (t < d) {
      int ai = offset * (2 * t + 1) - 1, bi = offset * (2 * t + 2) - 1;
      s[bi] += s[ai];
    }
    offset <<= 1;
  }
  __syncthreads();
  if (t == 0) {
    if (block_sums) block_sums[blockIdx.x] = s[SCAN_PER_BLOCK - 1];
    s[SCAN_PER_BLOCK - 1] = 0;
  }
  // down-sweep
  for (int d = 1; d < SCAN_PER_BLOCK; d <<= 1) {
    offset >>= 1;
    __syncthreads();
    if (t < d) {
      int ai = offset * (2 * t + 1) - 1, bi = offset * (2 * t + 2) - 1;
      int64_t v = s[ai];
      s[ai] = s[bi];
      s[bi] += v;
    }
  }
  __syncthreads();
  if (i0 < n) out[i0] = s[2 * t];
  if (i1 < n) out[i1] = s[2 * t + 1];
}

__global__ void k_scan_add(int64_t* out, int64_t n, const int64_t* block_offsets) {
  int64_t i = (int64_t)blockIdx.x * SCAN_PER_BLOCK + threadIdx.x;
  int64_t add = block_offsets[blockIdx.x];
  if (i < n) out[i] += add;
  if (i + SCAN_NT < n) out[i + SCAN_NT] += add;
}

__global__ void k_scan_total(const int64_t* out, const int64_t* in_last_val, int64_t n, int64_t* total) {
  *total = out[n - 1] + *in_last_val;
}

template <class In>
__global__ void k_last_value(const In* in, int64_t n, int64_t* dst) {
  *dst = (int64_t)in[n - 1];
}

template <class In>
int scan_impl(const In* d_in, int64_t* d_out, int64_t n, int64_t* total, cudaStream_t st) {
  if (n <= 0) {
    if (total) *total = 0;
    return RS_OK;
  }
  int64_t nb = (n + SCAN_PER_BLOCK - 1) / SCAN_PER_BLOCK;
  int64_t* sums = nullptr;
  int64_t* tmp = nullptr;
  RS_CUDA(cudaMallocAsync((void**)&tmp, 2 * sizeof(int64_t), st));
  // keep the last input value: d_out may alias d_in
  k_last_value<In><<<1, 1, 0, st>>>(d_in, n, tmp);
  RS_CHECK_LAUNCH();
  if (nb > 1) RS_CUDA(cudaMallocAsync((void**)&sums, nb * sizeof(int64_t), st));
  k_scan_blocks<In><<<(unsigned)nb, SCAN_NT, 0, st>>>(d_in, d_out, n, sums);
  RS_CHECK_LAUNCH();
  if (nb > 1) {
    int64_t dummy;
    RS_TRY(scan_impl<int64_t>(sums, sums, nb, &dummy, st));
    k_scan_add<<<(unsigned)nb, SCAN_NT, 0, st>>>(d_out, n, sums);
    RS_CHECK_LAUNCH();
  }
  k_scan_total<<<1, 1, 0, st>>>(d_out, tmp, n, tmp + 1);
  RS_CHECK_LAUNCH();
  if (total) {
    RS_CUDA(cudaMemcpyAsync(total, tmp + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaStreamSynchronize(st));
  }
  if (sums) RS_CUDA(cudaFreeAsync(sums, st));
  RS_CUDA(cudaFreeAsync(tmp, st));
  return RS_OK;
}

// ------------------------------------------------------------ radix sort
constexpr int RS_TILE = 256;       // elements per warp tile (8 chunks of 32)
constexpr int RS_WARPS = 4;        // warps (tiles) per block

__global__ void k_radix_hist(const uint64_t* keys, int n, int shift, int ntiles, int* counts) {
  __shared__ int h[RS_WARPS][256];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int tile = blockIdx.x * RS_WARPS + warp;
  for (int d = lane; d < 256; d += 32) h[warp][d] = 0;
  __syncwarp();
  if (tile < ntiles) {
    int base = tile * RS_TILE;
    for (int c = 0; c < RS_TILE; c += 32) {
      int i = base + c + lane;
      if (i < n) atomicAdd(&h[warp][(int)((keys[i] >> shift) & 255u)], 1);
    }
    __syncwarp();
    for (int d = lane; d < 256; d += 32) counts[(int64_t)d * ntiles + tile] = h[warp][d];
  }
}

__global__ void k_radix_scatter(const uint64_t* keys, const int* vals, uint64_t* ko, int* vo, int n,
                                int shift, int ntiles, const int64_t* offs) {
  __shared__ int64_t cnt[RS_WARPS][256];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int tile = blockIdx.x * RS_WARPS + warp;
  if (tile >= ntiles) return;
  for (int d = lane; d < 256; d += 32) cnt[warp][d] = offs[(int64_t)d * ntiles + tile];
  __syncwarp();
  unsigned lt = (1u << lane) - 1u;
  int base = tile * RS_TILE;
  for (int c = 0; c < RS_TILE; c += 32) {
    int i = base + c + lane;
    bool ok = i < n;
    int dg = ok ? (int)((keys[i] >> shift) & 255u) : 256 + lane;   // invalid lanes never match
    unsigned peers = __match_any_sync(0xffffffffu, dg);
    int rank = __popc(peers & lt);
    int64_t pos = ok ? cnt[warp][dg] + rank : 0;
    __syncwarp();
    if (ok) {
      ko[pos] = keys[i];
      vo[pos] = vals[i];
      if (rank == 0) cnt[warp][dg] += __popc(peers);
    }
    __syncwarp();
  }
}

__global__ void k_reduce_max(const int* in, int n, int* out) {
  __shared__ int s[1024];
  int m = -2147483647;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = max(m, in[i]);
  s[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s[threadIdx.x] = max(s[threadIdx.x], s[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

}  // namespace

int scan_i64(const int64_t* d_in, int64_t* d_out, int64_t n, int64_t* total, cudaStream_t st) {
  return scan_impl<int64_t>(d_in, d_out, n, total, st);
}

int scan_i32_to_i64(const int* d_in, int64_t* d_out, int64_t n, int64_t* total, cudaStream_t st) {
  return scan_impl<int>(d_in, d_out, n, total, st);
}

int radix_sort_pairs(uint64_t* keys, int* vals, uint64_t* keys_tmp, int* vals_tmp, int n, int bits,
                     cudaStream_t st) {
  if (n <= 1 || bits <= 0) return RS_OK;
  int ntiles = (n + RS_TILE - 1) / RS_TILE;
  int nblk = (ntiles + RS_WARPS - 1) / RS_WARPS;
  int* counts = nullptr;
  int64_t* offs = nullptr;
  RS_CUDA(cudaMallocAsync((void**)&counts, sizeof(int) * 256 * (size_t)ntiles, st));
  RS_CUDA(cudaMallocAsync((void**)&offs, sizeof(int64_t) * 256 * (size_t)ntiles, st));
  uint64_t* ka = keys;
  int* va = vals;
  uint64_t* kb = keys_tmp;
  int* vb = vals_tmp;
  int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    int shift = 8 * p;
    k_radix_hist<<<nblk, 32 * RS_WARPS, 0, st>>>(ka, n, shift, ntiles, counts);
    RS_CHECK_LAUNCH();
    RS_TRY(scan_impl<int>(counts, offs, (int64_t)256 * ntiles, nullptr, st));
    k_radix_scatter<<<nblk, 32 * RS_WARPS, 0, st>>>(ka, va, kb, vb, n, shift, ntiles, offs);
    RS_CHECK_LAUNCH();
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    RS_CUDA(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st));
    RS_CUDA(cudaMemcpyAsync(vals, va, sizeof(int) * n, cudaMemcpyDeviceToDevice, st));
  }
  RS_CUDA(cudaFreeAsync(counts, st));
  RS_CUDA(cudaFreeAsync(offs, st));
  return RS_OK;
}

int reduce_max_i32(const int* d_in, int n, int* out, cudaStream_t st) {
  if (n <= 0) {
    *out = 0;
    return RS_OK;
  }
  int* d = nullptr;
  RS_CUDA(cudaMallocAsync((void**)&d, sizeof(int), st));
  k_reduce_max<<<1, 1024, 0, st>>>(d_in, n, d);
  RS_CHECK_LAUNCH();
  RS_CUDA(cudaMemcpyAsync(out, d, sizeof(int), cudaMemcpyDeviceToHost, st));
  RS_CUDA(cudaStreamSynchronize(st));
  RS_CUDA(cudaFreeAsync(d, st));
  return RS_OK;
}

}  // namespace rs
