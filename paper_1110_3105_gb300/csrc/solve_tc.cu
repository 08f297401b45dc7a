// Multi-column solve on the tensor cores, operands fed by TMA.
//
// The same two-pass telescoping product as the persistent solve (eq.
// multilevel-inverse applied right to left, Sec. 4.3: upward u = calD b,
// c = calR b per box; the root; downward x = u + calL x_parent), for many
// right-hand sides in float arithmetic: the FP32 solve and the float forward
// operator of the refinement (eq. multilevel-compression with the stored
// blocks [D ; P] and P^T).  A work unit is 128 rows x TN columns of one box's
// block product on the tensor cores (tcgen05.mma kind::tf32, accumulator in
// tensor memory).  Every operand is kept as two tf32 values a = hi + lo and a
// product is formed as lo*hi + hi*lo + hi*hi (three MMAs per K step), about
// fp32 accuracy.  The factor rows are stored split; the vectors are stored as
// plain floats and split on their way in: the TMA copy lands in the hi slot
// of a stage and two converter warps rewrite it in place as hi and fill the
// lo slot before the MMAs read the stage.
//
// Data layout (per handle, per precision mode and column count):
//   * per tree depth d, float vectors of ldp_d rows x R columns; every box's
//     segment starts at a multiple of 32 rows (its padded offset poff), the
//     gaps stay zero; the input of the upward pass (v), calD b (u) and the
//     result of the downward pass (x) at depths above the leaves; the
//     leaves' input is the caller's B permuted to tree order by one streaming
//     kernel, and the leaves' result goes to the caller's X (double) through
//     the permutation;
//   * factor rows row-major with a 32-multiple row pitch per depth, hi and lo
//     arrays: the rows of [calD ; calR] (upward operand) and of calL
//     (downward operand, preceded by delta zero columns, delta = the
//     misalignment of the box's skeleton slot in its parent's vector mod 4,
//     so that the TMA copy of the parent's vector starts on a 16-byte
//     boundary and the extra rows meet zero factor columns);
//   * one 2D tensor map per array and depth (128-byte swizzle, box 32 K
//     elements x 128 rows or TN columns): a K chunk of a unit is four TMA
//     copies straight into the shared-memory layout the MMA reads.
//
// The CTA is warp-specialised: warp 0 (one thread) claims tiles in
// dependency order, waits for their inputs (bounded spin on the per-box
// counters) and issues the TMA copies of each K chunk into a ring of stages;
// warps 10-11 split each landed input chunk into its hi and lo parts; warp 1
// (one thread) issues the MMAs of each converted stage and releases it
// (tcgen05.commit), two tensor-memory accumulators alternating; warps 2-9
// read a finished accumulator (warp w: lanes 32 (w % 4)..), store the
// results, and publish a tile with one release-add on its counter.
// Every wait is bounded; past its limit a waiter raises the error flags and
// all roles drain and leave.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cuda/atomic>
#include <mutex>
#include <vector>

#include "rs_internal.h"
#include "tc.cuh"

namespace rs {

namespace {

constexpr int K_UP = 0, K_ROOT = 1, K_DOWN = 2;
constexpr int TT_NE = 256;            // 8 epilogue warps: two per tensor-memory lane quarter
constexpr int TT_NC = 64;             // 2 converter warps (warps 10, 11)
constexpr int TT_NT = 64 + TT_NE + TT_NC;   // + the producer warp and the MMA warp
constexpr int TT_TM = 128, TT_KC = 32;
constexpr int TT_POLLS = 1 << 30;
constexpr long long TT_WAIT_NS = 500000000;   // give up a stage / accumulator wait after 0.5 s
constexpr int TT_SPIN = 1 << 22;              // dependency spin limit (~0.4 s with the sleeps)
constexpr int TT_UQ = 8;
// Tensor maps per depth: A_up and A_dn (hi, lo) for copies of 32, 64 and 128
// factor rows, then V, X and U (hi, lo).
constexpr int NMAP = 18;
constexpr int M_AUP = 0, M_ADN = 6, M_V = 12, M_X = 14, M_U = 16;

// A tile with everything its producer and epilogue need, precomputed on
// the host (one load per tile instead of a chain of dependent lookups).
struct TTile {
  int g, r0, c0, c1, kind;
  int d, n, rows, nkc;
  int nk1;                     // K chunks from the first input (the rest: the second)
  int wait_idx, wait_target;   // counter (index into the counter array) and its per-epoch target (0: none)
  int sig_idx;                 // counter released when the tile is done
  int mapA, mapB, mapB2;       // tensor maps: factor rows (for this tile's copy height), inputs
  int ah;                      // factor rows copied per chunk (32, 64 or 128)
  int ay, bx, bx2;             // first factor row; first row of each input (multiples of 32)
  int64_t pos0;                // padded position of row r0 of the box in its depth's vectors
  int64_t slot;                // padded position of the skeletons in the parent's vectors
  int64_t off;                 // tree position of the box's first point (leaves)
};

struct TDev {
  const TTile* tiles;
  int ntiles;
  int L;
  const int* perm;
  float* const* uh;
  float* const* ul;
  float* const* xh;
  float* const* xl;
  float* const* vh;
  float* const* vl;
  const int64_t* ldp;
  const CUtensorMap* maps;   // NMAP per depth
  int R;                     // columns of every vector (chunk stride / 32)
  int Rr;                    // columns of this call (<= R); units past them are skipped
  int* dispatch;
  int* dflag;
  int* cnt;                  // dependency counters: per box, its children's upward tiles | its own downward tiles
  unsigned long long* trace;
};

struct TUnit {
  int t, c0, cw, nkc, last;
};

template <int TN> struct TCfg {
  static constexpr int NS = TN >= 256 ? 2 : TN >= 128 ? 3 : 4;   // stages within 227 KB
  static constexpr uint32_t a_bytes = TT_TM * 128;
  static constexpr uint32_t b_bytes = (uint32_t)TN * 128;
  static constexpr uint32_t stage = 2 * a_bytes + 2 * b_bytes;
  static constexpr size_t bytes = 1024 + (size_t)NS * stage;
  static constexpr uint32_t tmem_cols = 2 * TN;
};

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(tc::smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
                   tc::smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// 3D tiled TMA copy global -> shared of the box {32, rows, 1} at (0, y, z)
// (innermost coordinate always 0); completion counted in bytes on bar.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(tc::smem_u32(dst)),
      "l"(map), "r"(0), "r"(y), "r"(z), "r"(tc::smem_u32(bar))
      : "memory");
}
__device__ inline int ld_acquire(const int* p) {
  cuda::atomic_ref<const int, cuda::thread_scope_device> a(*p);
  return a.load(cuda::memory_order_acquire);
}
__device__ inline bool spin_until(const int* cnt, int target, int* flag, int* dflag) {
  int spins = 0;
  while (ld_acquire(cnt) < target) {
    if (++spins > TT_SPIN) {
      atomicExch(dflag, 1);
      atomicExch(flag, 1);
      return false;
    }
    if ((spins & 63) == 0 && *(volatile int*)dflag) return false;
    __nanosleep(64);
  }
  return true;
}
// Vectors are chunk-interleaved: the 32 rows pos = 32 z .. 32 z + 31 of all R
// columns are one contiguous block (column c at offset 32 c), so the K chunk
// of TN columns a unit reads is a single contiguous TN x 128-byte copy.
__host__ __device__ __forceinline__ int64_t vidx(int64_t pos, int64_t c, int64_t R) {
  return ((pos >> 5) * R + c) * 32 + (pos & 31);
}
__device__ __forceinline__ void split_store(float* hi, float* lo, int64_t i, float v) {
  float h, l;
  tc::tf32_split(v, h, l);
  hi[i] = h;
  lo[i] = l;
}

template <int TN>
__global__ void __launch_bounds__(TT_NT, 1) k_solve_tma(TDev p, const double* B, int64_t ldb, double* X, int64_t ldx,
                                                        const double* sub, int epoch, int* flag) {
  using C = TCfg<TN>;
  constexpr int NS = C::NS;
  extern __shared__ unsigned char tt_raw[];
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) uint64_t s_full[NS], s_conv[NS], s_empty[NS], s_accf[2], s_acce[2];
  __shared__ TUnit s_unit[TT_UQ];
  __shared__ int s_eok[2];
  __shared__ int s_end[NS];   // 1: the stage carries the producer's end marker (no copies)
  __shared__ int s_cok;       // the converters' wait for the current stage succeeded
  const uint32_t raw = tc::smem_u32(tt_raw);
  unsigned char* base = tt_raw + ((1024u - (raw & 1023u)) & 1023u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::tmem_alloc(&s_taddr, C::tmem_cols);
  if (tid == 32) {
    for (int i = 0; i < NS; ++i) {
      tc::mbar_init(&s_full[i], 1);
      tc::mbar_init(&s_conv[i], 1);
      tc::mbar_init(&s_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&s_accf[i], 1);
      tc::mbar_init(&s_acce[i], TT_NE);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_taddr;
  auto raise = [&]() {
    atomicExch(p.dflag, 1);
    atomicExch(flag, 1);
  };

  if (warp == 0) {
    // ------------------------------------------------ scheduler + TMA issue
    if (lane == 0) {
      int s = 0, u = 0;
      int next = atomicAdd(p.dispatch, 1);
      bool bad = false;
      while (!bad) {
        const int t = next;
        if (t >= p.ntiles) break;
        if (p.trace) p.trace[3 * (size_t)t] = gtime();
        const TTile tl = p.tiles[t];
        const bool ok = tl.wait_target == 0 || spin_until(p.cnt + tl.wait_idx, epoch * tl.wait_target, flag, p.dflag);
        if (!ok || *(volatile int*)p.dflag) break;
        next = atomicAdd(p.dispatch, 1);   // in flight while this tile's copies are issued
        if (p.trace) p.trace[3 * (size_t)t + 1] = gtime();
        const int cend = min(tl.c1, p.Rr);
        if (cend <= tl.c0) {   // no columns of this call: nothing to compute, publish at once
          cuda::atomic_ref<int, cuda::thread_scope_device> c(p.cnt[tl.sig_idx]);
          c.fetch_add(1, cuda::memory_order_release);
          if (p.trace) p.trace[3 * (size_t)t + 2] = gtime();
          continue;
        }
        const CUtensorMap* mA = p.maps + tl.mapA;
        const uint32_t tx = 2u * (uint32_t)tl.ah * 128u + C::b_bytes;
        for (int c0 = tl.c0; c0 < cend && !bad; c0 += TN, ++u) {
          for (int kc = 0; kc < tl.nkc; ++kc, ++s) {
            const int si = s % NS;
            if (!tc::mbar_wait(&s_empty[si], ((s / NS) & 1) ^ 1, TT_POLLS, TT_WAIT_NS)) {
              raise();
              bad = true;
              break;
            }
            if (kc == 0) s_unit[u % TT_UQ] = TUnit{t, c0, min(TN, cend - c0), tl.nkc, c0 + TN >= cend ? 1 : 0};
            unsigned char* st = base + (size_t)si * C::stage;
            s_end[si] = 0;
            mbar_expect_tx(&s_full[si], tx);
            // the first nk1 chunks of the input from one vector, the rest from
            // the second (down tiles: x_parent, then u); both bases are
            // multiples of 32 rows.  Factor rows past ah keep stale values:
            // they only reach accumulator rows the epilogue never stores.
            const bool first = kc < tl.nk1;
            const CUtensorMap* mB = p.maps + (first ? tl.mapB : tl.mapB2);
            const int zb = first ? (tl.bx >> 5) + kc : (tl.bx2 >> 5) + (kc - tl.nk1);
            tma_load_3d(st, mA, tl.ay, kc, &s_full[si]);
            tma_load_3d(st + C::a_bytes, mA + 1, tl.ay, kc, &s_full[si]);
            tma_load_3d(st + 2 * C::a_bytes, mB, c0, zb, &s_full[si]);   // plain floats into the hi slot
          }
        }
      }
      // end marker through the next stage (no copies: a plain arrival)
      const int si = s % NS;
      if (!tc::mbar_wait(&s_empty[si], ((s / NS) & 1) ^ 1, TT_POLLS, TT_WAIT_NS)) raise();
      s_unit[u % TT_UQ] = TUnit{-1, 0, 0, 0, 0};
      s_end[si] = 1;
      mbar_arrive(&s_full[si]);
    }
    __syncwarp();
  } else if (warp >= 2 + TT_NE / 32) {
    // ------------------------------------------------ input split (2 warps)
    // Each landed stage: the input chunk (TN x 32 floats, 128-byte swizzled;
    // the split is elementwise, so the layout does not matter) becomes its
    // tf32 hi part in place and its lo part in the lo slot; then the stage
    // is handed to the MMA warp.  The end marker is passed on unchanged.
    const int ct = tid - (64 + TT_NE);
    for (int s = 0;; ++s) {
      const int si = s % NS;
      if (ct == 0) {
        const bool ok = tc::mbar_wait(&s_full[si], (s / NS) & 1, TT_POLLS, TT_WAIT_NS);
        if (!ok) raise();
        s_cok = ok ? 1 : 0;
      }
      named_sync(3, TT_NC);   // the landed stage (or the failed wait) is seen by both warps
      const bool end = !s_cok || s_end[si];
      if (!end && !*(volatile int*)p.dflag) {
        float4* bh = reinterpret_cast<float4*>(base + (size_t)si * C::stage + 2 * C::a_bytes);
        float4* bl = reinterpret_cast<float4*>(base + (size_t)si * C::stage + 2 * C::a_bytes + C::b_bytes);
#pragma unroll 4
        for (int i = ct; i < (int)(C::b_bytes / 16); i += TT_NC) {
          const float4 v = bh[i];
          float4 h, l;
          tc::tf32_split(v.x, h.x, l.x);
          tc::tf32_split(v.y, h.y, l.y);
          tc::tf32_split(v.z, h.z, l.z);
          tc::tf32_split(v.w, h.w, l.w);
          bh[i] = h;
          bl[i] = l;
        }
        tc::fence_smem_to_async();   // generic-proxy writes, read next by the tensor cores
      }
      named_sync(3, TT_NC);
      if (ct == 0) mbar_arrive(&s_conv[si]);
      if (end) break;
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------- MMA issue
    if (lane == 0) {
      constexpr uint32_t IDESC = tc::idesc(tc::FMT_TF32, TT_TM, TN);
      int s = 0;
      for (int u = 0;; ++u) {
        if (!tc::mbar_wait(&s_conv[s % NS], (s / NS) & 1, TT_POLLS, TT_WAIT_NS)) {
          raise();
          break;
        }
        const TUnit un = s_unit[u % TT_UQ];
        const int a = u & 1;
        const bool free_acc = tc::mbar_wait(&s_acce[a], ((u >> 1) & 1) ^ 1, TT_POLLS, TT_WAIT_NS);
        if (!free_acc) raise();
        if (un.t < 0 || !free_acc) {   // hand the end marker to the epilogue
          mbar_arrive(&s_accf[a]);
          break;
        }
        tc::fence_after_sync();
        const uint32_t dt = tmem + (uint32_t)(a * TN);
        bool bad = false;
        for (int kc = 0; kc < un.nkc; ++kc, ++s) {
          const int si = s % NS;
          if (kc > 0 && !tc::mbar_wait(&s_conv[si], (s / NS) & 1, TT_POLLS, TT_WAIT_NS)) {
            raise();
            bad = true;
            break;
          }
          tc::fence_after_sync();
          const uint32_t ah = tc::smem_u32(base + (size_t)si * C::stage), al = ah + C::a_bytes;
          const uint32_t bh = ah + 2 * C::a_bytes, bl = bh + C::b_bytes;
#pragma unroll
          for (int ks = 0; ks < TT_KC / 8; ++ks) {
            const uint32_t o = 32u * ks;
            tc::mma_tf32(dt, tc::desc_sw128(al + o), tc::desc_sw128(bh + o), IDESC, kc > 0 || ks > 0);
            tc::mma_tf32(dt, tc::desc_sw128(ah + o), tc::desc_sw128(bl + o), IDESC, true);
            tc::mma_tf32(dt, tc::desc_sw128(ah + o), tc::desc_sw128(bh + o), IDESC, true);
          }
          tc::mma_commit(&s_empty[si]);
        }
        if (bad) {
          mbar_arrive(&s_accf[a]);
          break;
        }
        tc::mma_commit(&s_accf[a]);
      }
    }
    __syncwarp();
  } else {
    // -------------------------------------------------------------- epilogue
    const int ew = warp & 3;                 // tensor-memory lanes 32 ew .. 32 ew + 31
    const int jb = ((warp - 2) >> 2) * (TN / 2);   // this warp's half of the columns
    const int i = 32 * ew + lane;
    const bool leader = tid == 64;
    const int64_t R = p.R;
    for (int u = 0;; ++u) {
      const int a = u & 1;
      if (leader) {
        s_eok[a] = tc::mbar_wait(&s_accf[a], (u >> 1) & 1, TT_POLLS, TT_WAIT_NS) ? 1 : 0;
        if (!s_eok[a]) raise();
      }
      named_sync(1, TT_NE);
      if (!s_eok[a]) break;
      tc::fence_after_sync();
      const TUnit un = s_unit[u % TT_UQ];
      if (un.t < 0 || *(volatile int*)p.dflag) break;
      const TTile tl = p.tiles[un.t];
      const int d = tl.d, n = tl.n;
      const bool down = tl.kind == K_DOWN;
      const int r = tl.r0 + i;
      const bool rin = r < tl.rows;
      const bool to_x = rin && r < n && d == p.L && (down || tl.kind == K_ROOT);
      const int64_t dst = to_x ? (int64_t)p.perm[tl.off + r] : 0;
      const uint32_t lrow = tmem + (uint32_t)(a * TN) + ((uint32_t)(32 * ew) << 16);
      const int c0 = un.c0, cw = un.cw;
      const int64_t pos = tl.pos0 + i;
      float* const uhd = p.uh[d];
      float* const xhd = p.xh[d];
      float* const vhp = d > 0 ? p.vh[d - 1] : nullptr;
      const int64_t pp = tl.slot + (r - n);
      constexpr int JW = TN / 2 < 32 ? TN / 2 : 32;   // columns per batch
      for (int j0 = jb; j0 < jb + TN / 2; j0 += JW) {
        float acc[JW];
#pragma unroll
        for (int q = 0; q < JW; q += 16) tc::tmem_ld16(lrow + (uint32_t)(j0 + q), acc + q);
        tc::tmem_ld_wait();
        if (!rin || j0 >= cw) continue;
        const int jn = min(JW, cw - j0);
        const int64_t c = c0 + j0;
        if (to_x) {   // the caller's X (down tiles already hold u + calL x_parent)
          if (sub) {
            double sv[JW];
#pragma unroll
            for (int q = 0; q < JW; ++q) sv[q] = q < jn ? sub[dst + (c + q) * ldx] : 0.0;
#pragma unroll
            for (int q = 0; q < JW; ++q)
              if (q < jn) X[dst + (c + q) * ldx] = f32_to_f64(__fsub_rn(f64_to_f32_rn(sv[q]), acc[q]));
          } else {
#pragma unroll
            for (int q = 0; q < JW; ++q)
              if (q < jn) X[dst + (c + q) * ldx] = f32_to_f64(acc[q]);
          }
        } else if (down || tl.kind == K_ROOT) {   // x, for the children's copies
#pragma unroll
          for (int q = 0; q < JW; ++q)
            if (q < jn) xhd[vidx(pos, c + q, R)] = acc[q];
        } else if (r < n) {   // u = calD b: the down tile reads it as an input
#pragma unroll
          for (int q = 0; q < JW; ++q)
            if (q < jn) uhd[vidx(pos, c + q, R)] = acc[q];
        } else {   // c = calR b into the parent's input
#pragma unroll
          for (int q = 0; q < JW; ++q)
            if (q < jn) vhp[vidx(pp, c + q, R)] = acc[q];
        }
      }
      tc::fence_before_sync();
      mbar_arrive(&s_acce[a]);
      if (un.last) {
        // every epilogue thread's stores of the tile precede the barrier;
        // one release-add publishes them to the waiter that acquires it
        named_sync(2, TT_NE);
        if (leader) {
          cuda::atomic_ref<int, cuda::thread_scope_device> c(p.cnt[tl.sig_idx]);
          c.fetch_add(1, cuda::memory_order_release);
          if (p.trace) p.trace[3 * (size_t)un.t + 2] = gtime();
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_free(tmem, C::tmem_cols);
}

// The caller's B (double, original order) into the leaves' float input
// vectors (tree order, padded): one CTA per leaf box and 64 columns.
__global__ void k_tma_in(const double* B, int64_t ldb, int Rr, int64_t R, const int* perm, const int64_t* off,
                         const int64_t* poff, const int* n, float* vh, float* vl) {
  const int b = blockIdx.x, c0 = blockIdx.y * 64;
  const int nb = n[b];
  const int64_t o = off[b], po = poff[b];
  for (int e = threadIdx.x; e < nb * 64; e += blockDim.x) {
    const int r = e % nb, c = c0 + e / nb;
    if (c >= Rr) break;
    const double v = B[(int64_t)perm[o + r] + (int64_t)c * ldb];
    vh[vidx(po + r, c, R)] = f64_to_f32_rn(v);
    (void)vl;
  }
}

// Factor rows in the tensor-core layout, hi and lo parts, chunk-interleaved
// like the vectors: the 32 columns 32 z .. 32 z + 31 of all `nrows` rows of
// the depth form one block (row q at offset 32 q), zeros where a row has no
// entry; src is one box's column-major block of `rows` x `cols`, written from
// column `shift` on.
// One CTA per box and 32 source columns (blockIdx.y); consecutive threads
// take consecutive columns of one row, so their stores fall into one 128-byte
// chunk row; the column-strided reads of the source block are shared through
// the cache by the warps of neighbouring rows.
__global__ void k_tma_factors(const float* src, const int64_t* soff, const int* rows, const int* cols,
                              const int* shift, const int64_t* rb, int64_t nrows, float* hi, float* lo) {
  const int b = blockIdx.x, c0 = 32 * blockIdx.y;
  const int nr = rows[b], nc = cols[b], sh = shift ? shift[b] : 0;
  if (c0 >= nc) return;
  const int cw = min(32, nc - c0);
  const float* s = src + soff[b];
  for (int e = threadIdx.x; e < nr * cw; e += blockDim.x) {
    const int c = c0 + e % cw, r = e / cw;
    const int64_t k = sh + c;
    split_store(hi, lo, ((k >> 5) * nrows + rb[b] + r) * 32 + (k & 31), s[r + (int64_t)c * nr]);
  }
}

// The identity block of the downward factor rows: row r of a box gets a 1 in
// column c1 + r (c1 = the box's first column after its calL chunks), so the
// product with the input chunks [x_parent ; u] adds u (hi part exactly 1, lo
// part 0 from the zeroed array).
__global__ void k_tma_ident(const int64_t* rb, const int* n, const int* c1, int64_t nrows, float* hi) {
  const int b = blockIdx.x;
  for (int r = threadIdx.x; r < n[b]; r += blockDim.x) {
    const int64_t k = c1[b] + r;
    hi[((k >> 5) * nrows + rb[b] + r) * 32 + (k & 31)] = 1.0f;
  }
}

// ------------------------------------------------------------------ host
// Per handle: the padded geometry (computed once), the vectors per column
// bucket (64, 128, ..., 1024 columns; shared by the two modes, which run one
// after the other on a stream), the factor rows per mode, and one plan (tile
// list, counters, tensor maps) per (mode, column bucket, TN).  Every device
// buffer comes from the stream-ordered pool and goes back with the handle.
struct TGeo {
  int L = 0, G = 0;
  std::vector<int> gbase, depth, n, k, parent, delta, kpu, kpd;
  std::vector<int64_t> off, poff, slot, rbu, rbd, ldp, rows_up, rows_dn;
};

struct TVec {
  int R = 0;
  std::vector<float*> uh, ul, vh, vl, xh, xl;
};

struct TFac {
  int mode = -1;
  std::vector<float*> ahu, alu, ahd, ald;
};

struct TPlan {
  int mode = -1, R = 0, TN = 0;
  int ntiles = 0, nbox = 0;
  int* counters = nullptr;   // dispatch | device flag | per box: children's upward tiles | own downward tiles
  int epoch = 0;
  bool dirty = false;
  int* flag_host = nullptr;
  int* flag_dev = nullptr;
  TDev dev{};
  TVec* vec = nullptr;
  int nleaf = 0;
  const int64_t* leaf_off = nullptr;
  const int64_t* leaf_poff = nullptr;
  const int* leaf_n = nullptr;
  double bytes = 0, flops = 0;
  unsigned long long* trace = nullptr;   // per tile: claimed, inputs ready, published (ns)
  bool traced = false;
  std::vector<TTile> h_tiles;
};

struct TCache {
  TGeo geo;
  bool have_geo = false;
  std::vector<TVec*> vecs;
  std::vector<TFac*> facs;
  std::vector<TPlan*> plans;
  std::vector<void*> mem;
  std::vector<int*> flags;   // mapped pinned host words
  TPlan* last = nullptr;     // the plan of the last launch
};

std::mutex g_map_mu;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

int get_encode() {
  std::lock_guard<std::mutex> lk(g_map_mu);
  if (g_encode) return RS_OK;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return fail(RS_ERR_CUDA, "tensor-core solve: cuTensorMapEncodeTiled unavailable");
  }
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  return RS_OK;
}

// A chunk-interleaved float array as a 3D tensor {32, rows, chunks} (the 32
// elements of a row within a chunk contiguous, rows 128 bytes apart, chunks
// rows x 128 bytes apart); box {32, box_rows, 1}, 128-byte swizzle, zero
// fill out of bounds.
int make_map(CUtensorMap* m, const float* base, uint64_t rows, uint64_t chunks, uint32_t box_rows) {
  rows = std::max<uint64_t>(1, rows);
  const cuuint64_t dims[3] = {32, rows, std::max<uint64_t>(1, chunks)};
  const cuuint64_t strides[2] = {32 * sizeof(float), rows * 32 * sizeof(float)};
  const cuuint32_t box[3] = {32, box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(RS_ERR_CUDA, "tensor-core solve: tensor map encoding failed (%d)", (int)r);
  return RS_OK;
}

int cache_alloc(TCache* c, void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  if (cudaMallocAsync(p, std::max<size_t>(16, bytes), st) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(RS_ERR_OOM, "tensor-core solve: device allocation of %zu bytes failed", bytes);
  }
  c->mem.push_back(*p);
  return RS_OK;
}
template <class T>
int tup(TCache* c, T** d, const std::vector<T>& v, cudaStream_t st) {
  RS_TRY(cache_alloc(c, (void**)d, sizeof(T) * std::max<size_t>(1, v.size()), st));
  if (!v.empty()) RS_CUDA(cudaMemcpyAsync(*d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
  return RS_OK;
}
int talloc0(TCache* c, float** d, size_t count, cudaStream_t st) {
  RS_TRY(cache_alloc(c, (void**)d, sizeof(float) * std::max<size_t>(1, count), st));
  RS_CUDA(cudaMemsetAsync(*d, 0, sizeof(float) * std::max<size_t>(1, count), st));
  return RS_OK;
}

int64_t rup(int64_t a, int64_t m) { return (a + m - 1) / m * m; }

void make_geo(Handle* h, TGeo& g) {
  const int L = h->L;
  g.L = L;
  g.gbase.assign(L + 1, 0);
  int G = 0;
  for (int d = L; d >= 0; --d) {
    g.gbase[d] = G;
    G += h->lv[d].nbox;
  }
  g.G = G;
  g.depth.assign(G, 0);
  g.n.assign(G, 0);
  g.k.assign(G, 0);
  g.parent.assign(G, -1);
  g.delta.assign(G, 0);
  g.off.assign(G, 0);
  g.poff.assign(G, 0);
  g.slot.assign(G, 0);
  g.rbu.assign(G, 0);
  g.rbd.assign(G, 0);
  g.ldp.assign(L + 1, 0);
  g.rows_up.assign(L + 1, 0);
  g.rows_dn.assign(L + 1, 0);
  g.kpu.assign(L + 1, 32);
  g.kpd.assign(L + 1, 32);
  for (int d = 0; d <= L; ++d) {   // padded offsets and factor row bases per depth
    const Level& lv = h->lv[d];
    int64_t acc = 0, ru = 0, rd = 0;
    for (int b = 0; b < lv.nbox; ++b) {
      const int gi = g.gbase[d] + b;
      g.depth[gi] = d;
      g.n[gi] = lv.h_n[b];
      g.k[gi] = d > 0 ? lv.h_k[b] : 0;
      g.off[gi] = lv.h_off[b];
      g.parent[gi] = d > 0 ? g.gbase[d - 1] + lv.h_parent[b] : -1;
      g.poff[gi] = acc;
      acc += rup(std::max(1, g.n[gi]), 32);
      g.rbu[gi] = ru;
      ru += g.n[gi] + g.k[gi];
      g.rbd[gi] = rd;
      rd += d > 0 ? g.n[gi] : 0;
      g.kpu[d] = std::max<int>(g.kpu[d], (int)rup(g.n[gi], 32));
    }
    g.ldp[d] = std::max<int64_t>(32, acc);
    g.rows_up[d] = ru;
    g.rows_dn[d] = rd;
  }
  for (int d = 1; d <= L; ++d) {
    const Level& lv = h->lv[d];
    const Level& up = h->lv[d - 1];
    for (int b = 0; b < lv.nbox; ++b) {
      const int gi = g.gbase[d] + b;
      const int pb = lv.h_parent[b];
      g.slot[gi] = g.poff[g.gbase[d - 1] + pb] + (lv.h_skoff[b] - up.h_off[pb]);
      g.delta[gi] = (int)(g.slot[gi] & 31);   // the copy of the parent's vector starts at its chunk
      // x_parent chunks, then the identity block that adds u
      g.kpd[d] = std::max<int>(g.kpd[d], (int)(rup(g.k[gi] + g.delta[gi], 32) + rup(std::max(1, g.n[gi]), 32)));
    }
  }
}

int get_vec(TCache* c, int R, cudaStream_t st, TVec** out) {
  for (TVec* v : c->vecs)
    if (v->R == R) {
      *out = v;
      return RS_OK;
    }
  const TGeo& g = c->geo;
  TVec* v = new TVec();
  c->vecs.push_back(v);
  v->R = R;
  const int L = g.L;
  v->uh.assign(L + 1, nullptr);
  v->ul = v->vh = v->vl = v->xh = v->xl = v->uh;
  // every depth's vectors in one zeroed block (ldp is a multiple of 32 rows,
  // so every array starts 128-byte aligned); the vectors are plain floats,
  // split in shared memory, so the lo arrays are the hi arrays
  size_t total = 0;
  for (int d = 0; d <= L; ++d) total += (size_t)g.ldp[d] * R * (d < L ? 3 : 2);
  float* blk = nullptr;
  RS_TRY(talloc0(c, &blk, total, st));
  float* q = blk;
  for (int d = 0; d <= L; ++d) {
    const size_t vs = (size_t)g.ldp[d] * R;
    v->uh[d] = q; q += vs;
    v->vh[d] = q; q += vs;
    if (d < L) {
      v->xh[d] = q; q += vs;
    } else {   // never written or read at the leaves
      v->xh[d] = v->vh[d];
    }
    v->ul[d] = v->uh[d];
    v->vl[d] = v->vh[d];
    v->xl[d] = v->xh[d];
  }
  *out = v;
  return RS_OK;
}

int get_fac(Handle* h, TCache* c, int mode, cudaStream_t st, TFac** out) {
  for (TFac* f : c->facs)
    if (f->mode == mode) {
      *out = f;
      return RS_OK;
    }
  const TGeo& g = c->geo;
  TFac* f = new TFac();
  c->facs.push_back(f);
  f->mode = mode;
  const int L = g.L;
  f->ahu.assign(L + 1, nullptr);
  f->alu = f->ahd = f->ald = f->ahu;
  // the four factor-row arrays of every depth in one zeroed block
  std::vector<size_t> szu(L + 1), szd(L + 1);
  size_t total = 0;
  for (int d = 0; d <= L; ++d) {
    szu[d] = rup((int64_t)g.rows_up[d] * g.kpu[d], 64);
    szd[d] = rup(std::max<int64_t>(1, g.rows_dn[d]) * g.kpd[d], 64);
    total += 2 * (szu[d] + szd[d]);
  }
  float* blk = nullptr;
  RS_TRY(talloc0(c, &blk, total, st));
  {
    float* q = blk;
    for (int d = 0; d <= L; ++d) {
      f->ahu[d] = q; q += szu[d];
      f->alu[d] = q; q += szu[d];
      f->ahd[d] = q; q += szd[d];
      f->ald[d] = q; q += szd[d];
    }
  }
  // per-box tables of every depth, staged together and copied once
  struct Off {
    size_t ru, cu, su, bu, rd, cd, sd, bd, sh, c1;
    int cmax_u, cmax_d;
  };
  std::vector<Off> off(L + 1);
  HostPack pk;
  for (int d = 0; d <= L; ++d) {
    const Level& lv = h->lv[d];
    std::vector<int> ru(lv.nbox), cu(lv.nbox), rdn(lv.nbox), cdn(lv.nbox), sh(lv.nbox), c1(lv.nbox);
    std::vector<int64_t> su(lv.nbox), sd(lv.nbox), bu(lv.nbox), bd(lv.nbox);
    int cmax_u = 1, cmax_d = 1;
    for (int b = 0; b < lv.nbox; ++b) {
      const int gi = g.gbase[d] + b;
      ru[b] = g.n[gi] + g.k[gi];
      cu[b] = g.n[gi];
      su[b] = lv.h_uoff[b];
      bu[b] = g.rbu[gi];
      rdn[b] = g.n[gi];
      cdn[b] = g.k[gi];
      sd[b] = d > 0 ? lv.h_loff[b] : 0;
      bd[b] = g.rbd[gi];
      sh[b] = g.delta[gi];
      c1[b] = (int)rup(g.k[gi] + g.delta[gi], 32);
      cmax_u = std::max(cmax_u, cu[b]);
      cmax_d = std::max(cmax_d, cdn[b]);
    }
    Off& o = off[d];
    o.ru = pk.add(ru); o.cu = pk.add(cu); o.su = pk.add(su); o.bu = pk.add(bu);
    o.rd = pk.add(rdn); o.cd = pk.add(cdn); o.sd = pk.add(sd); o.bd = pk.add(bd);
    o.sh = pk.add(sh); o.c1 = pk.add(c1);
    o.cmax_u = cmax_u;
    o.cmax_d = cmax_d;
  }
  unsigned char* tb = nullptr;
  RS_TRY(tup(c, &tb, pk.buf, st));
  for (int d = 0; d <= L; ++d) {
    // sources: the FP32 solve's [calD ; calR] and calL, or the float forward
    // factors [D ; P] and Q^T
    const Level& lv = h->lv[d];
    const float* Us = (const float*)(mode == RS_PREC_FP32 ? lv.U32 : lv.FU32);
    const float* Ls = (const float*)(mode == RS_PREC_FP32 ? lv.Lf32 : lv.FL32);
    const Off& o = off[d];
    auto I32 = [&](size_t x) { return reinterpret_cast<const int*>(tb + x); };
    auto I64 = [&](size_t x) { return reinterpret_cast<const int64_t*>(tb + x); };
    k_tma_factors<<<dim3(lv.nbox, (o.cmax_u + 31) / 32), 256, 0, st>>>(Us, I64(o.su), I32(o.ru), I32(o.cu), nullptr,
                                                                        I64(o.bu), g.rows_up[d], f->ahu[d], f->alu[d]);
    RS_CHECK_LAUNCH();
    if (d > 0) {
      const int64_t nr = std::max<int64_t>(1, g.rows_dn[d]);
      k_tma_factors<<<dim3(lv.nbox, (o.cmax_d + 31) / 32), 256, 0, st>>>(Ls, I64(o.sd), I32(o.rd), I32(o.cd),
                                                                          I32(o.sh), I64(o.bd), nr, f->ahd[d],
                                                                          f->ald[d]);
      RS_CHECK_LAUNCH();
      k_tma_ident<<<lv.nbox, 128, 0, st>>>(I64(o.bd), I32(o.rd), I32(o.c1), nr, f->ahd[d]);
      RS_CHECK_LAUNCH();
    }
  }
  *out = f;
  return RS_OK;
}

int build_plan(Handle* h, TCache* c, int mode, int R, int TN, cudaStream_t st, TPlan** out) {
  RS_TRY(get_encode());
  if (!c->have_geo) {
    make_geo(h, c->geo);
    c->have_geo = true;
  }
  const TGeo& g = c->geo;
  TVec* vec = nullptr;
  TFac* fac = nullptr;
  RS_TRY(get_vec(c, R, st, &vec));
  RS_TRY(get_fac(h, c, mode, st, &fac));
  TPlan* P = new TPlan();
  c->plans.push_back(P);
  P->mode = mode;
  P->R = R;
  P->TN = TN;
  P->vec = vec;
  const int L = g.L, G = g.G;
  P->nbox = G;
  const std::vector<int>& n = g.n;
  const std::vector<int>& k = g.k;
  const std::vector<int>& parent = g.parent;
  std::vector<int> up_need(G, 0), dn_need(G, 0);
  // tiles in topological order, as the persistent solve lists them
  std::vector<TTile> tiles;
  const int nb = (R + TN - 1) / TN;
  auto col_ranges = [&](int d, bool dn) {
    const Level& lv = h->lv[d];
    int64_t rt = 0;
    for (int b = 0; b < lv.nbox; ++b)
      rt += ((dn ? lv.h_n[b] : lv.h_n[b] + (d > 0 ? lv.h_k[b] : 0)) + TT_TM - 1) / TT_TM;
    const int sp = (int)std::max<int64_t>(1, std::min<int64_t>(nb, 1024 / std::max<int64_t>(1, rt)));
    const int per = ((nb + sp - 1) / sp) * TN;
    std::vector<std::pair<int, int>> cr;
    for (int cc = 0; cc < R; cc += per) cr.push_back({cc, std::min(R, cc + per)});
    return cr;
  };
  // counters: cnt[2 + g] = upward tiles of g's children done, cnt[2 + G + g]
  // = g's own downward (root: root) tiles done
  auto mk = [&](int gi, int r0, std::pair<int, int> cr, int kind) {
    TTile t{};
    t.g = gi;
    t.r0 = r0;
    t.c0 = cr.first;
    t.c1 = cr.second;
    t.kind = kind;
    const int d = g.depth[gi];
    t.d = d;
    t.n = n[gi];
    t.rows = kind == K_DOWN ? n[gi] : n[gi] + k[gi];
    const int left = t.rows - r0;   // rows of this tile
    const int hsel = left <= 32 ? 0 : left <= 64 ? 1 : 2;
    t.ah = 32 << hsel;
    if (kind == K_DOWN) {
      t.nk1 = (int)(rup(k[gi] + g.delta[gi], 32) / 32);
      t.nkc = t.nk1 + (int)(rup(std::max(1, n[gi]), 32) / 32);
      t.wait_idx = 2 + G + parent[gi];
      t.mapA = NMAP * d + M_ADN + 2 * hsel;
      t.mapB = NMAP * (d - 1) + M_X;
      t.mapB2 = NMAP * d + M_U;
      t.ay = (int)(g.rbd[gi] + r0);
      t.bx = (int)(g.slot[gi] - g.delta[gi]);
      t.bx2 = (int)g.poff[gi];
      t.sig_idx = 2 + G + gi;
    } else {
      t.nkc = std::max(1, (n[gi] + TT_KC - 1) / TT_KC);
      t.nk1 = t.nkc;
      t.wait_idx = 2 + gi;
      t.mapA = NMAP * d + M_AUP + 2 * hsel;
      t.mapB = NMAP * d + M_V;
      t.mapB2 = t.mapB;
      t.ay = (int)(g.rbu[gi] + r0);
      t.bx = (int)g.poff[gi];
      t.bx2 = t.bx;
      t.sig_idx = kind == K_ROOT ? 2 + G + gi : 2 + parent[gi];
    }
    t.pos0 = g.poff[gi] + r0;
    t.slot = g.slot[gi];
    t.off = g.off[gi];
    return t;
  };
  for (int d = L; d >= 1; --d) {
    auto cr = col_ranges(d, false);
    for (int b = 0; b < h->lv[d].nbox; ++b) {
      const int gi = g.gbase[d] + b;
      for (int r0 = 0; r0 < n[gi] + k[gi]; r0 += TT_TM)
        for (auto& cc : cr) tiles.push_back(mk(gi, r0, cc, K_UP));
      up_need[parent[gi]] += (int)((n[gi] + k[gi] + TT_TM - 1) / TT_TM) * (int)cr.size();
    }
  }
  {
    auto cr = col_ranges(0, false);
    const int gi = g.gbase[0];
    for (int r0 = 0; r0 < n[gi]; r0 += TT_TM)
      for (auto& cc : cr) tiles.push_back(mk(gi, r0, cc, K_ROOT));
    dn_need[gi] = (int)((n[gi] + TT_TM - 1) / TT_TM) * (int)cr.size();
  }
  for (int d = 1; d <= L; ++d) {
    auto cr = col_ranges(d, true);
    for (int b = 0; b < h->lv[d].nbox; ++b) {
      const int gi = g.gbase[d] + b;
      for (int r0 = 0; r0 < n[gi]; r0 += TT_TM)
        for (auto& cc : cr) tiles.push_back(mk(gi, r0, cc, K_DOWN));
      dn_need[gi] = (int)((n[gi] + TT_TM - 1) / TT_TM) * (int)cr.size();
    }
  }
  for (TTile& t : tiles)   // per-epoch targets of the counters each tile waits on
    t.wait_target = t.kind == K_DOWN ? dn_need[parent[t.g]] : up_need[t.g];
  P->ntiles = (int)tiles.size();
  P->h_tiles = tiles;
  TDev& v = P->dev;
  v.ntiles = P->ntiles;
  v.L = L;
  v.R = R;
  v.Rr = R;
  v.perm = h->perm;
  // the plan's tables (tiles, leaf offsets, tensor maps, vector pointers,
  // counters) staged together and copied in one piece
  HostPack pk;
  const size_t o_tiles = pk.add(tiles);
  size_t o_lo = 0, o_lp = 0, o_ln = 0;
  {
    const int nl = h->lv[L].nbox;
    std::vector<int64_t> lo(nl), lp(nl);
    std::vector<int> ln(nl);
    for (int b = 0; b < nl; ++b) {
      lo[b] = g.off[g.gbase[L] + b];
      lp[b] = g.poff[g.gbase[L] + b];
      ln[b] = n[g.gbase[L] + b];
    }
    o_lo = pk.add(lo);
    o_lp = pk.add(lp);
    o_ln = pk.add(ln);
    P->nleaf = nl;
  }
  std::vector<CUtensorMap> maps((size_t)NMAP * (L + 1));
  for (int d = 0; d <= L; ++d) {
    CUtensorMap* m = maps.data() + (size_t)NMAP * d;
    const int64_t rdn = std::max<int64_t>(1, g.rows_dn[d]);
    for (int hs = 0; hs < 3; ++hs) {
      const uint32_t ah = 32u << hs;
      RS_TRY(make_map(m + M_AUP + 2 * hs, fac->ahu[d], g.rows_up[d], g.kpu[d] / 32, ah));
      RS_TRY(make_map(m + M_AUP + 2 * hs + 1, fac->alu[d], g.rows_up[d], g.kpu[d] / 32, ah));
      RS_TRY(make_map(m + M_ADN + 2 * hs, fac->ahd[d], rdn, g.kpd[d] / 32, ah));
      RS_TRY(make_map(m + M_ADN + 2 * hs + 1, fac->ald[d], rdn, g.kpd[d] / 32, ah));
    }
    const uint64_t ch = g.ldp[d] / 32;
    RS_TRY(make_map(m + M_V, vec->vh[d], R, ch, TN));
    RS_TRY(make_map(m + M_V + 1, vec->vl[d], R, ch, TN));
    RS_TRY(make_map(m + M_X, vec->xh[d], R, ch, TN));
    RS_TRY(make_map(m + M_X + 1, vec->xl[d], R, ch, TN));
    RS_TRY(make_map(m + M_U, vec->uh[d], R, ch, TN));
    RS_TRY(make_map(m + M_U + 1, vec->ul[d], R, ch, TN));
  }
  {
    const size_t o_maps = pk.add(maps);
    const size_t o_p0 = pk.add(vec->uh), o_p1 = pk.add(vec->ul), o_p2 = pk.add(vec->xh), o_p3 = pk.add(vec->xl),
                 o_p4 = pk.add(vec->vh), o_p5 = pk.add(vec->vl);
    std::vector<int> zeros(2 + 2 * (size_t)G, 0);
    const size_t o_cnt = pk.add(zeros);
    unsigned char* tb = nullptr;
    RS_TRY(tup(c, &tb, pk.buf, st));
    v.tiles = reinterpret_cast<const TTile*>(tb + o_tiles);
    P->leaf_off = reinterpret_cast<int64_t*>(tb + o_lo);
    P->leaf_poff = reinterpret_cast<int64_t*>(tb + o_lp);
    P->leaf_n = reinterpret_cast<int*>(tb + o_ln);
    v.maps = reinterpret_cast<const CUtensorMap*>(tb + o_maps);
    v.uh = reinterpret_cast<float* const*>(tb + o_p0);
    v.ul = reinterpret_cast<float* const*>(tb + o_p1);
    v.xh = reinterpret_cast<float* const*>(tb + o_p2);
    v.xl = reinterpret_cast<float* const*>(tb + o_p3);
    v.vh = reinterpret_cast<float* const*>(tb + o_p4);
    v.vl = reinterpret_cast<float* const*>(tb + o_p5);
    P->counters = reinterpret_cast<int*>(tb + o_cnt);
  }
  v.dispatch = P->counters;
  v.dflag = P->counters + 1;
  v.cnt = P->counters;
  v.trace = nullptr;
  RS_TRY(flag_take(&P->flag_host, &P->flag_dev));
  c->flags.push_back(P->flag_host);
  // algorithmic work per column: the float factors read once, B read and X
  // written (double), 2 flops per stored scalar
  double fa = 0.0;
  for (auto& lv : h->lv) fa += (double)lv.usz + (double)lv.lsz;
  P->bytes = 4.0 * fa;
  P->flops = 2.0 * fa;
  *out = P;
  return RS_OK;
}

template <int TN>
int launch_tn(Handle* h, TCache* c, TPlan* P, const double* B, int64_t ldb, int Rr, double* X, int64_t ldx,
              const double* sub, cudaStream_t st) {
  using C = TCfg<TN>;
  RS_CUDA(cudaFuncSetAttribute(k_solve_tma<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::bytes));
  int dev = 0, nsm = 0;
  RS_CUDA(cudaGetDevice(&dev));
  RS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int grid = std::max(1, std::min(nsm, P->ntiles));
  if (++P->epoch > (1 << 20) || P->dirty) {
    RS_CUDA(cudaMemsetAsync(P->counters, 0, sizeof(int) * (2 + 2 * (size_t)P->nbox), st));
    P->epoch = 1;
    P->dirty = false;
  }
  const int wait_epoch = take_wait_fault() ? P->epoch + 1 : P->epoch;
  RS_CUDA(cudaMemsetAsync(P->counters, 0, 2 * sizeof(int), st));
  *P->flag_host = 0;
  P->dev.Rr = Rr;
  P->dev.trace = nullptr;
  P->traced = false;
  if (prof_tiles_on()) {   // tile timeline for rs_profile_tiles
    if (!P->trace) RS_TRY(cache_alloc(c, (void**)&P->trace, sizeof(unsigned long long) * 3 * (size_t)P->ntiles, st));
    P->dev.trace = P->trace;
    P->traced = true;
  }
  prof_begin(prec_cat(P->mode), st);
  {
    dim3 gin(P->nleaf, (Rr + 63) / 64);
    k_tma_in<<<gin, 256, 0, st>>>(B, ldb, Rr, P->R, h->perm, P->leaf_off, P->leaf_poff, P->leaf_n,
                                  P->vec->vh[h->L], P->vec->vl[h->L]);
    RS_CHECK_LAUNCH();
  }
  k_solve_tma<TN><<<grid, TT_NT, C::bytes, st>>>(P->dev, B, ldb, X, ldx, sub, wait_epoch, P->flag_dev);
  RS_CHECK_LAUNCH();
  prof_end(prec_cat(P->mode), st, P->bytes + 2.0 * 8.0 * (double)h->N * Rr, P->flops * Rr);
  return RS_OK;
}

}  // namespace

// Column buckets of the tensor-core plans: one plan serves every column
// count up to its bucket.
int tc_bucket(int R) {
  int b = 64;
  while (b < R) b <<= 1;
  return b;
}

int solve_tc_run(Handle* h, int mode, int TN, const double* B, int64_t ldb, int R, double* X, int64_t ldx,
                 const double* sub, cudaStream_t st) {
  if (h->cplx || (mode != RS_PREC_FP32 && mode != MODE_FWD_F32) || (TN != 64 && TN != 128 && TN != 256) || R < 1 ||
      R > TC_MAX_COLS)
    return fail(RS_ERR_ARG, "tensor-core solve: real kernels, float modes, TN in {64, 128, 256}, 1..%d columns",
                TC_MAX_COLS);
  if (!h->pers_tc) h->pers_tc = new TCache();
  TCache* c = (TCache*)h->pers_tc;
  const int Rb = std::max(tc_bucket(R), TN);
  TPlan* P = nullptr;
  for (TPlan* q : c->plans)
    if (q->mode == mode && q->R == Rb && q->TN == TN) P = q;
  if (!P) RS_TRY(build_plan(h, c, mode, Rb, TN, st, &P));
  c->last = P;
  switch (TN) {
    case 64: return launch_tn<64>(h, c, P, B, ldb, R, X, ldx, sub, st);
    case 128: return launch_tn<128>(h, c, P, B, ldb, R, X, ldx, sub, st);
    default: return launch_tn<256>(h, c, P, B, ldb, R, X, ldx, sub, st);
  }
}

int tc_tile_trace(Handle* h, int mode, int R, int64_t cap, int* kind, int* depth, int* r0, int* ncol,
                  double* t_claim, double* t_start, double* t_end, int64_t* count) {
  TCache* c = (TCache*)h->pers_tc;
  TPlan* P = c ? c->last : nullptr;
  if (!P || P->mode != mode || P->R != std::max(tc_bucket(R), P->TN) || !P->traced) return RS_ERR_STATE;
  std::vector<unsigned long long> tr(3 * (size_t)P->ntiles);
  RS_CUDA(cudaDeviceSynchronize());
  RS_CUDA(cudaMemcpy(tr.data(), P->trace, sizeof(unsigned long long) * tr.size(), cudaMemcpyDeviceToHost));
  unsigned long long t0 = ~0ull;
  for (int t = 0; t < P->ntiles; ++t) t0 = std::min(t0, tr[3 * (size_t)t]);
  const int64_t n = std::min<int64_t>(cap, P->ntiles);
  for (int64_t t = 0; t < n; ++t) {
    const TTile& tl = P->h_tiles[t];
    if (kind) kind[t] = tl.kind;
    if (depth) depth[t] = tl.d;
    if (r0) r0[t] = tl.r0;
    if (ncol) ncol[t] = tl.c1 - tl.c0;
    if (t_claim) t_claim[t] = 1e-3 * (double)(tr[3 * t] - t0);
    if (t_start) t_start[t] = 1e-3 * (double)(tr[3 * t + 1] - t0);
    if (t_end) t_end[t] = 1e-3 * (double)(tr[3 * t + 2] - t0);
  }
  if (count) *count = P->ntiles;
  return RS_OK;
}

// A later non-tensor-core launch makes the tensor-core timeline stale for
// rs_profile_tiles.
void tc_forget_last(Handle* h) {
  TCache* c = (TCache*)h->pers_tc;
  if (c) c->last = nullptr;
}

int tc_check(Handle* h) {
  TCache* c = (TCache*)h->pers_tc;
  if (!c) return RS_OK;
  int rc = RS_OK;
  for (TPlan* P : c->plans)
    if (P->flag_host && *(volatile int*)P->flag_host) {
      P->dirty = true;
      *P->flag_host = 0;
      rc = RS_ERR_TIMEOUT;
    }
  if (rc != RS_OK) return fail(RS_ERR_TIMEOUT, "tensor-core solve: a wait ran out (flag set by the device)");
  return RS_OK;
}

// Called with the device idle (handle destruction).
void free_tc(Handle* h) {
  TCache* c = (TCache*)h->pers_tc;
  if (!c) return;
  for (void* m : c->mem) cudaFreeAsync(m, 0);
  for (int* f : c->flags) flag_release(f);
  for (TPlan* P : c->plans) delete P;
  for (TVec* v : c->vecs) delete v;
  for (TFac* f : c->facs) delete f;
  delete c;
  h->pers_tc = nullptr;
}

}  // namespace rs
