// Persistent, dependency-driven solve: the whole upward pass, the root and
// the downward pass (eq. multilevel-inverse applied right to left, Sec. 4.3)
// in one kernel launch.
//
// Work is cut into tiles of at most 32 rows x CT columns of one box's block
// product:
//   up tile    rows of [calD ; calR] b   (box b of depth d >= 1; its rows
//              beyond n land in the parent's input vector)
//   root tile  rows of calS^-1 c          (depth 0)
//   down tile  rows of u + calL x_parent  (depth d >= 1)
// Tiles are listed in topological order (leaves first, then up to the root,
// then down to the leaves) and handed out to warps by an atomic counter, so a
// warp only ever waits on tiles that were handed out before its own and are
// being worked on by resident warps.  A box's up tiles wait until every up
// tile of its children has finished (one counter per box); a down tile waits
// until every down (or root) tile of its parent has finished.  Counters grow
// monotonically across solves (target = epoch * count), waits are bounded
// spins: past the limit a warp sets the error flag and leaves, and so in turn
// does every warp waiting on it.
//
// Lanes own rows (column-major factors -> coalesced loads); every lane keeps
// CT accumulators for the tile's columns; the right-hand-side rows of the box
// are staged 32 at a time in per-warp shared memory.  The per-depth vectors
// are column-major (one column per right-hand side), so staging loads and
// result stores are coalesced along the rows.  Leaf tiles read B and write X
// in the caller's order through the tree permutation.
#include <algorithm>
#include <map>
#include <tuple>
#include <mutex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cuda/atomic>
#include <vector>

#include "rs_internal.h"
#include "tc.cuh"

namespace rs {

namespace {

constexpr int P_NT = 256;
constexpr int TC_TM = 128;   // rows of a tensor-core tile (solve_tc.cu)
constexpr int P_WARPS = P_NT / 32;
constexpr int MAX_SPIN = 1 << 22;

enum TileKind { T_UP = 0, T_ROOT = 1, T_DOWN = 2 };

struct Tile {
  int g;      // global box index
  int r0;     // first row
  int c0;     // columns [c0, c1)
  int c1;
  int kind;
};

// Per global box (all depths concatenated, leaves first).
struct BoxTab {
  int* depth;
  int* n;
  int* k;
  int64_t* off;
  int64_t* skoff;
  int64_t* uoff;
  int64_t* loff;
  int* parent;      // global index of the parent (-1 for the root)
  int* up_need;     // up tiles of all children
  int* dn_need;     // own down tiles (root: root tiles)
};

template <class S>
struct Plan {
  const Tile* tiles;
  int ntiles;
  BoxTab bt;
  int L;
  const int* perm;
  S* const* v;          // per depth: input of the up pass (v[L] unused: B is read directly)
  S* const* u;          // per depth: calD b, then x
  const int64_t* ldv;   // per depth: leading dimension of v and u (column-major, ntot of the depth)
  const S* const* U;    // per depth factors
  const S* const* Lf;
  int* dispatch;
  int* dflag;           // device copy of the timeout flag (checked per tile)
  int* up_cnt;
  int* dn_cnt;
  unsigned long long* trace;   // per tile: claimed, dependencies met, done (ns); null unless profiling
};

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ inline int ld_acquire(const int* p) {
  cuda::atomic_ref<const int, cuda::thread_scope_device> a(*p);
  return a.load(cuda::memory_order_acquire);
}

// One thread waits until *cnt >= target; returns false (and raises both
// flags: the device one every warp polls, the host-mapped one the caller
// reads) on timeout.
__device__ inline bool spin_until(const int* cnt, int target, int* flag, int* dflag) {
  int spins = 0;
  while (ld_acquire(cnt) < target) {
    if (++spins > MAX_SPIN) {
      atomicExch(dflag, 1);
      atomicExch(flag, 1);
      return false;
    }
    if ((spins & 63) == 0 && *(volatile int*)dflag) return false;   // another waiter gave up
    __nanosleep(100);
  }
  return true;
}

// Lane 0 of the warp waits (spin_until); the verdict is broadcast.
__device__ inline bool wait_at_least(const int* cnt, int target, int* flag, int* dflag) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) ok = spin_until(cnt, target, flag, dflag) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
}

__device__ inline void signal(int* cnt) {
  __threadfence();
  __syncwarp();
  if ((threadIdx.x & 31) == 0) atomicAdd(cnt, 1);
}

// Ask L2 for the lines of a factor column segment (rows r, stride ld, count
// q) while a tile still waits for its inputs: the rows come from HBM once
// the wait ends instead of on the tile's critical path.
template <class S>
__device__ __forceinline__ void prefetch_rows(const S* col, size_t ld, int count) {
  for (int q = 0; q < count; ++q) asm volatile("prefetch.global.L2 [%0];" ::"l"(col + (size_t)q * ld));
}
// Whether a dependency counter has reached its target (one lane's look).
__device__ __forceinline__ bool ready(const int* cnt, int target) { return ld_acquire(cnt) >= target; }

template <class S> __device__ inline S ldcg(const S* p) { return __ldcg(p); }
template <> __device__ inline c128 ldcg<c128>(const c128* p) {
  double2 t = __ldcg(reinterpret_cast<const double2*>(p));
  return c128(t.x, t.y);
}
template <> __device__ inline c64 ldcg<c64>(const c64* p) {
  float2 t = __ldcg(reinterpret_cast<const float2*>(p));
  return c64(t.x, t.y);
}
template <> __device__ inline dfloat ldcg<dfloat>(const dfloat* p) {
  float2 t = __ldcg(reinterpret_cast<const float2*>(p));
  return dfloat(t.x, t.y);
}
template <> __device__ inline cdfloat ldcg<cdfloat>(const cdfloat* p) {
  float4 t = __ldcg(reinterpret_cast<const float4*>(p));
  return cdfloat(dfloat(t.x, t.y), dfloat(t.z, t.w));
}

// Read-only (non-coherent) loads for the factors, which no kernel writes
// during a solve.
template <class S> __device__ inline S ldro(const S* p) { return __ldg(p); }
template <> __device__ inline c128 ldro<c128>(const c128* p) {
  double2 t = __ldg(reinterpret_cast<const double2*>(p));
  return c128(t.x, t.y);
}
template <> __device__ inline c64 ldro<c64>(const c64* p) {
  float2 t = __ldg(reinterpret_cast<const float2*>(p));
  return c64(t.x, t.y);
}
template <> __device__ inline dfloat ldro<dfloat>(const dfloat* p) {
  float2 t = __ldg(reinterpret_cast<const float2*>(p));
  return dfloat(t.x, t.y);
}
template <> __device__ inline cdfloat ldro<cdfloat>(const cdfloat* p) {
  float4 t = __ldg(reinterpret_cast<const float4*>(p));
  return cdfloat(dfloat(t.x, t.y), dfloat(t.z, t.w));
}

template <class D, class S> __device__ inline D cv(S v) { return D(v); }
template <> __device__ inline float cv<float, double>(double v) { return f64_to_f32_rn(v); }
template <> __device__ inline double cv<double, float>(float v) { return f32_to_f64(v); }
template <> __device__ inline c64 cv<c64, c128>(c128 v) { return c64((float)v.re, (float)v.im); }
template <> __device__ inline c128 cv<c128, c64>(c64 v) { return c128((double)v.re, (double)v.im); }

// acc[c] += sum_{q < qn} col[q * ld] * stage[q][c] for one 32-column chunk.
// All factor loads of the chunk are issued before the FMAs (QB at a time)
// so a lane keeps up to QB loads in flight instead of one per iteration; the
// staged row stage[q][0..CT) is read with 128-bit loads (every lane reads the
// same address, so each load is one broadcast wavefront).
template <class S, int CT>
struct StageRow {
  __device__ static void fma(S* acc, S a, const S* row) {
#pragma unroll
    for (int c = 0; c < CT; ++c) acc[c] += a * row[c];
  }
};
template <int CT>
struct StageRow<float, CT> {
  __device__ static void fma(float* acc, float a, const float* row) {
    if (CT % 4 == 0) {
      const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
      for (int c = 0; c < CT / 4; ++c) {
        const float4 v = r4[c];
        acc[4 * c] += a * v.x;
        acc[4 * c + 1] += a * v.y;
        acc[4 * c + 2] += a * v.z;
        acc[4 * c + 3] += a * v.w;
      }
    } else {
#pragma unroll
      for (int c = 0; c < CT; ++c) acc[c] += a * row[c];
    }
  }
};
template <int CT>
struct StageRow<double, CT> {
  __device__ static void fma(double* acc, double a, const double* row) {
    if (CT % 2 == 0) {
      const double2* r2 = reinterpret_cast<const double2*>(row);
#pragma unroll
      for (int c = 0; c < CT / 2; ++c) {
        const double2 v = r2[c];
        acc[2 * c] += a * v.x;
        acc[2 * c + 1] += a * v.y;
      }
    } else {
#pragma unroll
      for (int c = 0; c < CT; ++c) acc[c] += a * row[c];
    }
  }
};

template <int CT>
struct StageRow<dfloat, CT> {
  __device__ static void fma(dfloat* acc, dfloat a, const dfloat* row) {
    if (CT % 2 == 0) {
      const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
      for (int c = 0; c < CT / 2; ++c) {
        const float4 v = r4[c];
        df_fma(acc[2 * c], a, dfloat(v.x, v.y));
        df_fma(acc[2 * c + 1], a, dfloat(v.z, v.w));
      }
    } else {
#pragma unroll
      for (int c = 0; c < CT; ++c) df_fma(acc[c], a, row[c]);
    }
  }
};

template <int CT>
struct StageRow<cdfloat, CT> {
  __device__ static void fma(cdfloat* acc, cdfloat a, const cdfloat* row) {
#pragma unroll
    for (int c = 0; c < CT; ++c) cdf_fma(acc[c], a, row[c]);
  }
};

// Right-hand-side entries into the working type (integer-instruction
// conversions for float and double-float, see rs_common.cuh).
template <class S, class SIO> __device__ __forceinline__ S in_cv(SIO v) { return cv<S, SIO>(v); }
template <> __device__ __forceinline__ float in_cv<float, double>(double v) { return f64_to_f32_rn(v); }
template <> __device__ __forceinline__ dfloat in_cv<dfloat, double>(double v) { return f64_to_df(v); }
template <> __device__ __forceinline__ cdfloat in_cv<cdfloat, c128>(c128 v) {
  return cdfloat(f64_to_df(v.re), f64_to_df(v.im));
}

// Leaf output: the value itself, or sub - value (forward operator used for a
// residual b - A x).  In float and double-float the subtraction is done in
// the working type and the result, whose leading bits cancelled, is
// returned rounded to float precision relative to itself.
template <class S, class SIO> __device__ __forceinline__ SIO out_cv(const SIO* sub, int64_t i, S y) {
  const SIO v = cv<SIO, S>(y);
  return sub ? sub[i] - v : v;
}
template <> __device__ __forceinline__ double out_cv<float, double>(const double* sub, int64_t i, float y) {
  return f32_to_f64(sub ? __fsub_rn(f64_to_f32_rn(sub[i]), y) : y);
}
template <> __device__ __forceinline__ double out_cv<dfloat, double>(const double* sub, int64_t i, dfloat y) {
  if (sub) return f32_to_f64((f64_to_df(sub[i]) + (-y)).hi);
  return __dadd_rn(f32_to_f64(y.hi), f32_to_f64(y.lo));
}
template <> __device__ __forceinline__ c128 out_cv<cdfloat, c128>(const c128* sub, int64_t i, cdfloat y) {
  if (sub) {
    const c128 s = sub[i];
    return c128(f32_to_f64((f64_to_df(s.re) + (-y.re)).hi), f32_to_f64((f64_to_df(s.im) + (-y.im)).hi));
  }
  return c128(__dadd_rn(f32_to_f64(y.re.hi), f32_to_f64(y.re.lo)), __dadd_rn(f32_to_f64(y.im.hi), f32_to_f64(y.im.lo)));
}

template <class S, int CT>
__device__ __forceinline__ void chunk_fma(const S* col, size_t ld, int qn, const S* stage, S* acc) {
  constexpr int QB = CT == 1 ? 32 : (CT <= 8 ? 16 : 8);
  for (int q0 = 0; q0 < qn; q0 += QB) {
    S a[QB];
#pragma unroll
    for (int j = 0; j < QB; ++j) a[j] = (q0 + j < qn) ? ldro(col + (size_t)(q0 + j) * ld) : S(0.0);
#pragma unroll
    for (int j = 0; j < QB; ++j) StageRow<S, CT>::fma(acc, a[j], stage + (size_t)(q0 + j) * CT);
  }
}

// TR: record the tile timeline (a separate instantiation: the timer reads
// constrain instruction scheduling even when not taken).
template <class S, class SIO, int CT, bool TR>
__global__ void __launch_bounds__(P_NT) k_solve_pers(Plan<S> p, const SIO* B, int64_t ldb, SIO* X, int64_t ldx,
                                                     const SIO* sub, int R, int epoch, int* flag) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  S* stage = reinterpret_cast<S*>(smem) + (size_t)warp * 32 * CT;   // [32][CT]
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(p.dispatch, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= p.ntiles) break;
    if (*(volatile int*)p.dflag) return;   // another warp gave up waiting: leave too
    if (TR && lane == 0) p.trace[3 * (size_t)t] = gtime();
    const Tile tl = p.tiles[t];
    const int g = tl.g;
    const int d = p.bt.depth[g];
    const int n = p.bt.n[g], k = p.bt.k[g];
    const int64_t off = p.bt.off[g];

    if (tl.kind != T_DOWN) {
      // ---- up / root tile: rows of U b, U = [calD ; calR] ((n+k) x n)
      if (p.bt.up_need[g] > 0) {
        const int target = epoch * p.bt.up_need[g];
        int wait = 0;
        if (lane == 0) wait = !ready(&p.up_cnt[g], target);
        if (__shfl_sync(0xffffffffu, wait, 0) && CT == 1 && tl.r0 + lane < n + k)
          prefetch_rows(p.U[d] + p.bt.uoff[g] + tl.r0 + lane, (size_t)(n + k), n);
        if (!wait_at_least(&p.up_cnt[g], target, flag, p.dflag)) return;
      }
      if (TR && lane == 0) p.trace[3 * (size_t)t + 1] = gtime();
      const int rows = n + k;
      const int r = tl.r0 + lane;
      const S* Ub = p.U[d] + p.bt.uoff[g];
      const bool leaf = d == p.L;
      const S* vin = leaf ? nullptr : p.v[d];
      const int64_t ldd = p.ldv[d];
      for (int c0 = tl.c0; c0 < tl.c1; c0 += CT) {
        const int cw = min(CT, tl.c1 - c0);
        S acc[CT];
#pragma unroll
        for (int c = 0; c < CT; ++c) acc[c] = S(0.0);
        for (int q0 = 0; q0 < n; q0 += 32) {
          const int qn = min(32, n - q0);
          if (lane >= qn) {   // rows past the chunk end stay zero (chunk_fma reads them times 0)
#pragma unroll
            for (int c = 0; c < CT; ++c) stage[lane * CT + c] = S(0.0);
          } else {
            const int64_t pos = off + q0 + lane;
            if (leaf) {
              const int64_t src = p.perm[pos];
#pragma unroll
              for (int c = 0; c < CT; ++c)
                stage[lane * CT + c] = c < cw ? in_cv<S, SIO>(B[src + (int64_t)(c0 + c) * ldb]) : S(0.0);
            } else {
#pragma unroll
              for (int c = 0; c < CT; ++c)
                stage[lane * CT + c] = c < cw ? ldcg(vin + (int64_t)(c0 + c) * ldd + pos) : S(0.0);
            }
          }
          __syncwarp();
          if (r < rows) chunk_fma<S, CT>(Ub + r + (size_t)q0 * rows, (size_t)rows, qn, stage, acc);
          __syncwarp();
        }
        if (r < rows) {
          if (r < n && tl.kind == T_ROOT && d == p.L) {   // single-box tree: the root is the answer
            const int64_t dst = p.perm[off + r];
#pragma unroll
            for (int c = 0; c < CT; ++c)
              if (c < cw) {
                const int64_t i = dst + (int64_t)(c0 + c) * ldx;
                X[i] = out_cv<S, SIO>(sub, i, acc[c]);
              }
          } else if (r < n) {
            S* uo = p.u[d] + (int64_t)c0 * ldd + off + r;
#pragma unroll
            for (int c = 0; c < CT; ++c)
              if (c < cw) uo[(int64_t)c * ldd] = acc[c];
          } else {
            const int64_t ldp = p.ldv[d - 1];
            S* vo = p.v[d - 1] + (int64_t)c0 * ldp + p.bt.skoff[g] + (r - n);
#pragma unroll
            for (int c = 0; c < CT; ++c)
              if (c < cw) vo[(int64_t)c * ldp] = acc[c];
          }
        }
      }
      if (tl.kind == T_ROOT) signal(&p.dn_cnt[g]);
      else signal(&p.up_cnt[p.bt.parent[g]]);
      if (TR && lane == 0) p.trace[3 * (size_t)t + 2] = gtime();
    } else {
      // ---- down tile: rows of u + calL x_parent (n x k)
      const int par = p.bt.parent[g];
      {
        const int target = epoch * p.bt.dn_need[par];
        int wait = 0;
        if (lane == 0) wait = !ready(&p.dn_cnt[par], target);
        if (__shfl_sync(0xffffffffu, wait, 0) && CT == 1 && tl.r0 + lane < n)
          prefetch_rows(p.Lf[d] + p.bt.loff[g] + tl.r0 + lane, (size_t)n, k);
        if (!wait_at_least(&p.dn_cnt[par], target, flag, p.dflag)) return;
      }
      if (TR && lane == 0) p.trace[3 * (size_t)t + 1] = gtime();
      const int r = tl.r0 + lane;
      const S* Lb = p.Lf[d] + p.bt.loff[g];
      const int64_t ldd = p.ldv[d], ldp = p.ldv[d - 1];
      const S* xpar = p.u[d - 1] + p.bt.skoff[g];
      for (int c0 = tl.c0; c0 < tl.c1; c0 += CT) {
        const int cw = min(CT, tl.c1 - c0);
        S acc[CT];
#pragma unroll
        for (int c = 0; c < CT; ++c) acc[c] = S(0.0);
        for (int q0 = 0; q0 < k; q0 += 32) {
          const int qn = min(32, k - q0);
#pragma unroll
          for (int c = 0; c < CT; ++c)
            stage[lane * CT + c] = (lane < qn && c < cw) ? ldcg(xpar + (int64_t)(c0 + c) * ldp + q0 + lane) : S(0.0);
          __syncwarp();
          if (r < n) chunk_fma<S, CT>(Lb + r + (size_t)q0 * n, (size_t)n, qn, stage, acc);
          __syncwarp();
        }
        if (r < n) {
          S* uo = p.u[d] + (int64_t)c0 * ldd + off + r;
          if (d == p.L) {
            const int64_t dst = p.perm[off + r];
#pragma unroll
            for (int c = 0; c < CT; ++c)
              if (c < cw) {
                const int64_t i = dst + (int64_t)(c0 + c) * ldx;
                X[i] = out_cv<S, SIO>(sub, i, ldcg(uo + (int64_t)c * ldd) + acc[c]);
              }
          } else {
#pragma unroll
            for (int c = 0; c < CT; ++c)
              if (c < cw) uo[(int64_t)c * ldd] = ldcg(uo + (int64_t)c * ldd) + acc[c];
          }
        }
      }
      signal(&p.dn_cnt[g]);
      if (TR && lane == 0) p.trace[3 * (size_t)t + 2] = gtime();
    }
  }
}


// ------------------------------------------------------------- CTA tiles
// Many right-hand sides: the same tile list and dependency counters, but a
// tile is a TM-row x TN-column block of one box's product computed by a
// whole CTA as a small register-blocked GEMM.  Factor and input chunks (32
// deep) are staged in shared memory with coalesced loads (the factor along
// its rows, the inputs along their column-major rows); every thread
// accumulates an RPT x CPT block and a warp owns TM / 4 consecutive rows, so
// warps past the box's last row skip the arithmetic; the result block is
// transposed through shared memory so that its stores are coalesced along the
// rows as well.
constexpr int C_NT = 128, C_TK = 32;
static_assert(C_TK == 32, "input staging maps a warp onto the 32 rows of a chunk");

// Thread layout of a TM x TN tile: CG column groups of CPT columns, the rest
// row groups of RPT rows; a warp owns TM / 4 consecutive rows.
template <int TM, int TN> struct CtaShape {
  static constexpr int CG = TN >= 64 ? 16 : 8;
  static constexpr int CPT = TN / CG;
  static constexpr int RPT = TM * CG / C_NT;
};

template <class S> __device__ __forceinline__ void mac(S& acc, S a, S b) { acc += a * b; }
template <> __device__ __forceinline__ void mac<dfloat>(dfloat& acc, dfloat a, dfloat b) { df_fma(acc, a, b); }
template <> __device__ __forceinline__ void mac<cdfloat>(cdfloat& acc, cdfloat a, cdfloat b) { cdf_fma(acc, a, b); }

// N consecutive elements from 16-byte aligned shared memory.
template <class S, int N> struct Lds {
  __device__ static void run(const S* p, S* o) {
#pragma unroll
    for (int i = 0; i < N; ++i) o[i] = p[i];
  }
};
template <int N> struct Lds<float, N> {
  __device__ static void run(const float* p, float* o) {
    static_assert(N % 2 == 0, "even vector");
    if constexpr (N % 4 == 0) {
#pragma unroll
      for (int i = 0; i < N / 4; ++i) {
        const float4 v = reinterpret_cast<const float4*>(p)[i];
        o[4 * i] = v.x; o[4 * i + 1] = v.y; o[4 * i + 2] = v.z; o[4 * i + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int i = 0; i < N / 2; ++i) {
        const float2 v = reinterpret_cast<const float2*>(p)[i];
        o[2 * i] = v.x; o[2 * i + 1] = v.y;
      }
    }
  }
};
template <int N> struct Lds<dfloat, N> {
  __device__ static void run(const dfloat* p, dfloat* o) {
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const float4 v = reinterpret_cast<const float4*>(p)[i];
      o[2 * i] = dfloat(v.x, v.y);
      o[2 * i + 1] = dfloat(v.z, v.w);
    }
  }
};
template <int N> struct Lds<double, N> {
  __device__ static void run(const double* p, double* o) {
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const double2 v = reinterpret_cast<const double2*>(p)[i];
      o[2 * i] = v.x; o[2 * i + 1] = v.y;
    }
  }
};

template <class S, int TM, int TN>
struct CtaSmem {
  static constexpr int BP = TN + 16 / (int)sizeof(S);   // padded input row (keeps 16-byte alignment)
  static constexpr int OP = TM + 1;                     // padded output column
  static constexpr int BSZ = C_TK * BP > TN * OP ? C_TK * BP : TN * OP;
  static constexpr size_t bytes = sizeof(S) * (size_t)(C_TK * TM + BSZ);
};

template <class S, class SIO, int TM, int TN>
__global__ void __launch_bounds__(C_NT) k_solve_cta(Plan<S> p, const SIO* B, int64_t ldb, SIO* X, int64_t ldx,
                                                    const SIO* sub, int epoch, int* flag) {
  using Sh = CtaShape<TM, TN>;
  constexpr int RPT = Sh::RPT, CPT = Sh::CPT, CG = Sh::CG;
  constexpr int BP = CtaSmem<S, TM, TN>::BP, OP = CtaSmem<S, TM, TN>::OP;
  constexpr int C_TM = TM;
  static_assert((C_NT / CG) * RPT == TM && CG * CPT == TN, "tile shape");
  static_assert((32 / CG) * RPT == TM / 4, "a warp owns TM / 4 rows");
  extern __shared__ __align__(16) unsigned char smem[];
  S* As = reinterpret_cast<S*>(smem);   // [TK][TM]
  S* Bs = As + C_TK * C_TM;             // [TK][BP]; the output block [TN][OP] reuses it
  __shared__ int s_tile, s_ok;
  const int tid = threadIdx.x;
  const int tx = tid % CG, ty = tid / CG;
  const int wrow = (tid >> 5) * (TM / 4);   // first row of this warp's rows
  // Thread 0 claims the next tile while the CTA works on the current one (the
  // list is topological, so a claimed tile never precedes one it waits on).
  int next = 0;
  if (tid == 0) next = atomicAdd(p.dispatch, 1);
  for (;;) {
    if (tid == 0) {
      const int t = next;
      int ok = 1;
      if (t < p.ntiles) {
        if (p.trace) p.trace[3 * (size_t)t] = gtime();
        const Tile tl = p.tiles[t];
        if (tl.kind != T_DOWN) {
          if (p.bt.up_need[tl.g] > 0)
            ok = spin_until(&p.up_cnt[tl.g], epoch * p.bt.up_need[tl.g], flag, p.dflag);
        } else {
          const int par = p.bt.parent[tl.g];
          ok = spin_until(&p.dn_cnt[par], epoch * p.bt.dn_need[par], flag, p.dflag);
        }
        if (ok) next = atomicAdd(p.dispatch, 1);
        if (p.trace) p.trace[3 * (size_t)t + 1] = gtime();
      }
      s_tile = t;
      s_ok = ok;
    }
    __syncthreads();
    const int t = s_tile;
    if (t >= p.ntiles || !s_ok) return;
    const Tile tl = p.tiles[t];
    const int g = tl.g;
    const int d = p.bt.depth[g];
    const int n = p.bt.n[g], k = p.bt.k[g];
    const int64_t off = p.bt.off[g];
    const bool down = tl.kind == T_DOWN;
    const int rows = down ? n : n + k;     // the root has k = 0
    const int K = down ? k : n;
    const S* A = down ? p.Lf[d] + p.bt.loff[g] : p.U[d] + p.bt.uoff[g];
    const bool leaf_in = !down && d == p.L;
    const S* vin = down ? p.u[d - 1] : (leaf_in ? nullptr : p.v[d]);
    const int64_t ldin = down ? p.ldv[d - 1] : p.ldv[d];
    const int64_t in0 = down ? p.bt.skoff[g] : off;
    const int r0 = tl.r0;
    const bool busy = wrow < rows - r0;    // warp-uniform
    // Stages (column block, k chunk) in order; float tiles load the next
    // stage's factor and input values into registers while the current one
    // is computed (software pipelining), the others load at staging time.  A
    // single-chunk factor block is staged once for all column blocks.
    constexpr bool PF = std::is_same<S, float>::value;
    constexpr int AN = C_TM * C_TK / C_NT, BN = C_TK * TN / C_NT;
    const int nkc = (K + C_TK - 1) / C_TK;
    const int ncb = (tl.c1 - tl.c0 + TN - 1) / TN;
    const int nstage = ncb * (nkc > 0 ? nkc : 1);
    const int ia = tid % C_TM, ka = tid / C_TM;   // A element (row ia, chunk rows ka + k AN-stride)
    const int kb = tid % C_TK, jb = tid / C_TK;   // B element (chunk row kb, columns jb + j * (C_NT / C_TK))
    int64_t bsrc_k0 = -1;                         // chunk start the B source index below belongs to
    int64_t bsrc = 0;
    S aR[PF ? AN : 1], bR[PF ? BN : 1];
    auto a_needed = [&](int st) { return nkc > 1 || st / nkc == 0; };
    auto b_source = [&](int k0) {   // input row of this thread's chunk row
      if (bsrc_k0 != k0) {
        bsrc_k0 = k0;
        const int kk = k0 + kb;
        bsrc = kk < K ? (leaf_in ? (int64_t)p.perm[off + kk] : in0 + kk) : -1;
      }
      return bsrc;
    };
    auto a_val = [&](int k0, int q) -> S {
      const int kk = ka + q * (C_NT / C_TM);
      return (r0 + ia < rows && k0 + kk < K) ? ldro(A + (r0 + ia) + (size_t)(k0 + kk) * rows) : S(0.0);
    };
    auto b_val = [&](int c0, int64_t src, int q) -> S {
      const int j = jb + q * (C_NT / C_TK);
      if (src < 0 || c0 + j >= tl.c1) return S(0.0);
      return leaf_in ? in_cv<S, SIO>(B[src + (int64_t)(c0 + j) * ldb]) : ldcg(vin + (int64_t)(c0 + j) * ldin + src);
    };
    auto prefetch = [&](int st) {
      if constexpr (PF) {
        const int k0 = (st % nkc) * C_TK, c0 = tl.c0 + (st / nkc) * TN;
        if (a_needed(st)) {
#pragma unroll
          for (int q = 0; q < AN; ++q) aR[q] = a_val(k0, q);
        }
        const int64_t src = b_source(k0);
#pragma unroll
        for (int q = 0; q < BN; ++q) bR[q] = b_val(c0, src, q);
      }
    };
    S acc[RPT][CPT];
    if (nkc > 0) prefetch(0);
    for (int st = 0; st < nstage; ++st) {
      const int cb = nkc > 0 ? st / nkc : st, kc = nkc > 0 ? st % nkc : 0;
      const int c0 = tl.c0 + cb * TN;
      const int cw = min(TN, tl.c1 - c0);
      if (kc == 0) {
#pragma unroll
        for (int a = 0; a < RPT; ++a)
#pragma unroll
          for (int b = 0; b < CPT; ++b) acc[a][b] = S(0.0);
      }
      if (nkc > 0) {
        const int k0 = kc * C_TK, kn = min(C_TK, K - k0);
        __syncthreads();   // the previous stage (or tile) is done with As / Bs
        if (a_needed(st)) {
#pragma unroll
          for (int q = 0; q < AN; ++q) As[(ka + q * (C_NT / C_TM)) * C_TM + ia] = PF ? aR[q] : a_val(k0, q);
        }
        {
          const int64_t src = PF ? 0 : b_source(k0);
#pragma unroll
          for (int q = 0; q < BN; ++q) Bs[kb * BP + jb + q * (C_NT / C_TK)] = PF ? bR[q] : b_val(c0, src, q);
        }
        __syncthreads();
        if (st + 1 < nstage) prefetch(st + 1);   // in flight while this stage computes
        if (busy) {
          for (int kk = 0; kk < kn; ++kk) {
            S a[RPT], b[CPT];
            Lds<S, RPT>::run(As + kk * C_TM + ty * RPT, a);
            Lds<S, CPT>::run(Bs + kk * BP + tx * CPT, b);
#pragma unroll
            for (int x = 0; x < RPT; ++x)
#pragma unroll
              for (int y = 0; y < CPT; ++y) mac(acc[x][y], a[x], b[y]);
          }
        }
      }
      if (nkc > 0 && kc < nkc - 1) continue;
    __syncthreads();   // every thread is done reading As / Bs
    S* Os = Bs;
    if (busy) {
#pragma unroll
      for (int x = 0; x < RPT; ++x)
#pragma unroll
        for (int y = 0; y < CPT; ++y) Os[(tx * CPT + y) * OP + ty * RPT + x] = acc[x][y];
    }
    __syncthreads();
    {
      const int i = tid % C_TM;
      const int r = r0 + i;
      const int j0 = tid / C_TM;
      constexpr int JS = C_NT / C_TM;
      if (r < rows) {
        if (!down) {
          if (r < n && tl.kind == T_ROOT && d == p.L) {   // single-box tree: the root is the answer
            const int64_t dst = p.perm[off + r];
            for (int j = j0; j < cw; j += JS) {
              const int64_t idx = dst + (int64_t)(c0 + j) * ldx;
              X[idx] = out_cv<S, SIO>(sub, idx, Os[j * OP + i]);
            }
          } else if (r < n) {
            const int64_t ld = p.ldv[d];
            S* uo = p.u[d] + (int64_t)c0 * ld + off + r;
            for (int j = j0; j < cw; j += JS) uo[(int64_t)j * ld] = Os[j * OP + i];
          } else {
            const int64_t ld = p.ldv[d - 1];
            S* vo = p.v[d - 1] + (int64_t)c0 * ld + p.bt.skoff[g] + (r - n);
            for (int j = j0; j < cw; j += JS) vo[(int64_t)j * ld] = Os[j * OP + i];
          }
        } else {
          const int64_t ld = p.ldv[d];
          S* uo = p.u[d] + (int64_t)c0 * ld + off + r;
          if (d == p.L) {
            const int64_t dst = p.perm[off + r];
            for (int j = j0; j < cw; j += JS) {
              const int64_t idx = dst + (int64_t)(c0 + j) * ldx;
              X[idx] = out_cv<S, SIO>(sub, idx, ldcg(uo + (int64_t)j * ld) + Os[j * OP + i]);
            }
          } else {
            for (int j = j0; j < cw; j += JS) uo[(int64_t)j * ld] = ldcg(uo + (int64_t)j * ld) + Os[j * OP + i];
          }
        }
      }
    }
    }   // stages
    // every thread's stores of this tile precede the barrier; thread 0's
    // release add publishes them to the waiter that acquires the counter
    __syncthreads();
    if (tid == 0) {
      cuda::atomic_ref<int, cuda::thread_scope_device> c(tl.kind == T_UP ? p.up_cnt[p.bt.parent[g]] : p.dn_cnt[g]);
      c.fetch_add(1, cuda::memory_order_release);
      if (p.trace) p.trace[3 * (size_t)t + 2] = gtime();
    }
  }
}


// ------------------------------------------------------------------- host
struct PersPlan {
  int prec = -1, R = 0, CT = 0;
  int TN = 0;                // > 0: CTA-tile kernel with TM x TN tiles
  int TM = 32;
  int ntiles = 0, nbox = 0;
  Tile* tiles = nullptr;
  BoxTab bt{};
  int* counters = nullptr;   // dispatch | device flag | up_cnt[G] | dn_cnt[G]
  int epoch = 0;
  void** ptrs = nullptr;     // v[L+1] | u[L+1] | U[L+1] | Lf[L+1]
  int64_t* ldv = nullptr;    // per depth ntot (leading dimension of v and u)
  int* flag_host = nullptr;  // mapped pinned
  int* flag_dev = nullptr;
  int grid = 0;              // CTAs of the launch (all resident)
  int occ = 0, nsm = 0;      // resident CTAs per SM at full occupancy, SM count
  int cps = 0;               // CTAs per SM of the current grid (0: full occupancy)
  int work_gen = -1;         // generation of the work buffers captured in ptrs
  unsigned long long* trace = nullptr;   // tile timeline of the last profiled launch (3 per tile)
  bool traced = false;
  std::vector<Tile> h_tiles;             // host copy of the tile list
  std::vector<int> h_depth;              // depth per global box
  bool dirty = false;        // a wait timed out: counters must restart
  std::vector<void*> mem;
};

struct PersCache {
  std::vector<PersPlan*> plans;
};

// Launch configurations chosen by the autotuner, shared by every handle of
// the process: (mode, column bucket, complex, N) -> tile * 16 + cps, the
// bucket being the column count rounded down to a power of two (a serving
// loop's batches of varying width share one tuning).
struct TuneKey {
  int mode, R, cplx;
  int64_t N;
  bool operator<(const TuneKey& o) const {
    return std::tie(mode, R, cplx, N) < std::tie(o.mode, o.R, o.cplx, o.N);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;

// Candidate tiles of the CTA kernel for R right-hand sides, as rows * 1000 +
// columns (0: the warp kernel, which suits few columns).  The first solve of
// a plan with several candidates times each and keeps the fastest (the
// summation order inside a tile is the same for every shape, so so are the
// results).  RS_SOLVE_TILE fixes the choice ("TMxTN" with TM, TN in
// {32, 64}; "0" forces the warp kernel).
// A launch configuration is tile * 16 + cps, cps the CTAs per SM (0: as
// many as fit).  Few columns use the warp kernel, whose dependency chain is
// the whole cost: fewer resident warps poll the dependency counters less
// and can shorten it, so its candidates vary cps.
std::vector<int> launch_configs(int R, bool tc) {
  static const int forced = [] {
    const char* e = getenv("RS_SOLVE_TILE");
    if (!e) return -1;
    int tm = 0, tn = 0;
    if (sscanf(e, "%dx%d", &tm, &tn) == 2 && (tm == 32 || tm == 64) && (tn == 32 || tn == 64)) return tm * 1000 + tn;
    if (sscanf(e, "%dx%d", &tm, &tn) == 2 && tm == 128 && (tn == 64 || tn == 128 || tn == 256)) return tm * 1000 + tn;
    return 0;
  }();
  if (forced == 0) return {0 * 16 + 0};
  if (forced > 0 && forced / 1000 == TC_TM && !tc) return {(R < 16 ? 0 : 32064) * 16};
  if (forced > 0) return {(R < 16 ? 0 : forced) * 16};
  if (R < 32) return {0 * 16 + 0, 0 * 16 + 3, 0 * 16 + 2};
  std::vector<int> c = R < 64 ? std::vector<int>{32032 * 16, 64032 * 16}
                              : std::vector<int>{32064 * 16, 32032 * 16, 64064 * 16};
  if (tc) {   // tensor-core tiles (float arithmetic, real kernels)
    c.push_back(128064 * 16);
    if (R > 64) c.push_back(128128 * 16);
    if (R > 128) c.push_back(128256 * 16);
  }
  return c;
}

// The tensor cores accumulate a block product in fp32 one K step after
// another: on blocks thousands deep (the 3D top levels) that loses about an
// order of magnitude against the CUDA-core FMA chains (1e-5 against 1e-6
// relative at N = 4096 on the sphere), which the refinement's float residual
// update cannot afford.  Tensor-core tiles therefore serve trees whose
// largest block is at most 320 deep (every 2D workload).
bool tc_shallow(const Handle* h) {
  int m = 0;
  for (const auto& lv : h->lv) m = std::max(m, lv.maxn);
  return m <= 320;
}

// Tensor-core tiles are candidates unless RS_SOLVE_TC=0.
bool tc_enabled() {
  static const bool on = [] {
    const char* e = getenv("RS_SOLVE_TC");
    return !(e && e[0] == '0');
  }();
  return on;
}

int ct_for(bool cplx, int prec, int R) {
  if (R == 1) return 1;
  if (R <= 8) return 8;
  if (prec == RS_PREC_FP64 || prec == MODE_FWD_DF) return cplx ? 8 : 16;
  return cplx ? 16 : 32;
}

}  // namespace

// Host staging of several small tables for one device block: each at a
// 256-byte aligned offset.
size_t HostPack::add_bytes(const void* p, size_t bytes) {
  const size_t o = (buf.size() + 255) & ~(size_t)255;
  buf.resize(o + std::max<size_t>(bytes, 1));
  if (bytes) std::memcpy(buf.data() + o, p, bytes);
  return o;
}

// The flag pool: pages of 256 mapped, portable pinned ints, never returned
// to the driver (a handful of pages serve a process).
namespace {
std::mutex g_flag_mu;
std::vector<int*> g_flag_free;
}  // namespace

int flag_take(int** host, int** dev) {
  int* f = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_flag_mu);
    if (g_flag_free.empty()) {
      int* page = nullptr;
      if (cudaHostAlloc((void**)&page, 256 * sizeof(int), cudaHostAllocMapped | cudaHostAllocPortable) !=
          cudaSuccess) {
        cudaGetLastError();
        return fail(RS_ERR_OOM, "pinned flag page allocation failed");
      }
      for (int i = 255; i >= 0; --i) g_flag_free.push_back(page + i);
    }
    f = g_flag_free.back();
    g_flag_free.pop_back();
  }
  *(volatile int*)f = 0;
  if (cudaHostGetDevicePointer((void**)dev, f, 0) != cudaSuccess) {
    cudaGetLastError();
    flag_release(f);
    return fail(RS_ERR_CUDA, "pinned flag: no device address");
  }
  *host = f;
  return RS_OK;
}

void flag_release(int* host) {
  if (!host) return;
  std::lock_guard<std::mutex> lk(g_flag_mu);
  g_flag_free.push_back(host);
}

namespace {

template <class T>
int dev_upload(PersPlan* P, T** d, const std::vector<T>& v, cudaStream_t st) {
  RS_CUDA(cudaMalloc((void**)d, sizeof(T) * std::max<size_t>(1, v.size())));
  P->mem.push_back(*d);
  if (!v.empty()) RS_CUDA(cudaMemcpyAsync(*d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
  return RS_OK;
}

// The tensor-core tiles (solve_tc.cu) exist for float arithmetic with
// double input and output: the FP32 solve and the float forward operator of
// real kernels.
template <class S, class SIO> struct TcOk { static constexpr bool value = false; };
template <> struct TcOk<float, double> { static constexpr bool value = true; };

template <class S, class SIO, int CT, int TM, int TN>
int launch_pers(Handle* h, PersPlan* P, const SIO* B, int64_t ldb, int R, SIO* X, int64_t ldx, const SIO* sub,
                cudaStream_t st) {
  constexpr int TMv = TN ? TM : 32, TNv = TN ? TN : 32;
  const size_t smem = TN ? CtaSmem<S, TMv, TNv>::bytes : sizeof(S) * 32 * CT * P_WARPS;
  const int nt = TN ? C_NT : P_NT;
  const void* fn = TN ? (const void*)k_solve_cta<S, SIO, TMv, TNv> : (const void*)k_solve_pers<S, SIO, CT, false>;
  if (smem > 48 * 1024) RS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (P->occ == 0) {
    int dev = 0;
    RS_CUDA(cudaGetDevice(&dev));
    RS_CUDA(cudaDeviceGetAttribute(&P->nsm, cudaDevAttrMultiProcessorCount, dev));
    RS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&P->occ, fn, nt, smem));
    P->occ = std::max(P->occ, 1);
  }
  {
    const int per_block = TN ? 1 : P_WARPS;   // tiles a block works on at once
    const int cps = P->cps > 0 ? std::min(P->cps, P->occ) : P->occ;
    P->grid = std::max(1, std::min(P->nsm * cps, div_up(P->ntiles, per_block)));
  }
  if (++P->epoch > (1 << 20) || P->dirty) {   // counters restart (overflow guard, or after a timeout)
    RS_CUDA(cudaMemsetAsync(P->counters, 0, sizeof(int) * (2 + 2 * (size_t)P->nbox), st));
    P->epoch = 1;
    P->dirty = false;
  }
  // injected fault: wait for one more round of tiles than will ever finish
  const int wait_epoch = take_wait_fault() ? P->epoch + 1 : P->epoch;
  RS_CUDA(cudaMemsetAsync(P->counters, 0, 2 * sizeof(int), st));   // dispatch and device flag
  Plan<S> pl;
  pl.tiles = P->tiles;
  pl.ntiles = P->ntiles;
  pl.bt = P->bt;
  pl.L = h->L;
  pl.perm = h->perm;
  const int L1 = h->L + 1;
  pl.v = (S* const*)P->ptrs;
  pl.u = (S* const*)(P->ptrs + L1);
  pl.U = (const S* const*)(P->ptrs + 2 * L1);
  pl.Lf = (const S* const*)(P->ptrs + 3 * L1);
  pl.ldv = P->ldv;
  pl.dispatch = P->counters;
  pl.dflag = P->counters + 1;
  pl.up_cnt = P->counters + 2;
  pl.dn_cnt = P->counters + 2 + P->nbox;
  pl.trace = nullptr;
  P->traced = false;
  if (prof_tiles_on()) {   // tile timeline for rs_profile_tiles
    if (!P->trace) {
      RS_CUDA(cudaMalloc((void**)&P->trace, sizeof(unsigned long long) * 3 * (size_t)P->ntiles));
      P->mem.push_back(P->trace);
    }
    pl.trace = P->trace;
    P->traced = true;
  }
  *P->flag_host = 0;
  prof_begin(prec_cat(P->prec), st);
  if constexpr (TN > 0) {
    k_solve_cta<S, SIO, TMv, TNv><<<P->grid, C_NT, smem, st>>>(pl, B, ldb, X, ldx, sub, wait_epoch, P->flag_dev);
  } else {
    if (pl.trace)
      k_solve_pers<S, SIO, CT, true><<<P->grid, P_NT, smem, st>>>(pl, B, ldb, X, ldx, sub, R, wait_epoch, P->flag_dev);
    else
      k_solve_pers<S, SIO, CT, false><<<P->grid, P_NT, smem, st>>>(pl, B, ldb, X, ldx, sub, R, wait_epoch,
                                                                   P->flag_dev);
  }
  RS_CHECK_LAUNCH();
  double sS = sizeof(S), fac = 0.0;
  for (auto& lv : h->lv) fac += (double)lv.usz + (double)lv.lsz;
  prof_end(prec_cat(P->prec), st, sS * fac + (double)R * h->N * 2.0 * sizeof(SIO),
           2.0 * (is_cplx<S>::value ? 4.0 : 1.0) * fac * R);
  return RS_OK;
}

}  // namespace

int prec_cat(int prec) {
  return prec == RS_PREC_FP64 ? P_SOLVE64 : prec == RS_PREC_FP32 ? P_SOLVE32 : P_RESID;
}

void free_pers(Handle* h) {
  free_tc(h);
  PersCache* c = (PersCache*)h->pers;
  if (!c) return;
  for (PersPlan* P : c->plans) {
    for (void* m : P->mem) cudaFree(m);
    flag_release(P->flag_host);
    delete P;
  }
  delete c;
  h->pers = nullptr;
}

// Device pointer table of a plan: the work vectors (which may have been
// regrown for a larger R since the plan was made) and the factors.
static int refresh_ptrs(Handle* h, PersPlan* P, cudaStream_t st) {
  const int L = h->L;
  const Handle::Work& w = h->work[P->prec];
  std::vector<void*> ptrs(4 * (L + 1));
  for (int d = 0; d <= L; ++d) {
    ptrs[d] = w.v[d];
    ptrs[(L + 1) + d] = w.u[d];
    const Level& lv = h->lv[d];
    void* const Us[4] = {lv.U, lv.U32, lv.FU32, lv.FUdf};
    void* const Ls[4] = {lv.Lf, lv.Lf32, lv.FL32, lv.FLdf};
    ptrs[2 * (L + 1) + d] = Us[P->prec];
    ptrs[3 * (L + 1) + d] = Ls[P->prec];
  }
  if (!P->ptrs) {
    RS_CUDA(cudaMalloc((void**)&P->ptrs, sizeof(void*) * ptrs.size()));
    P->mem.push_back(P->ptrs);
  }
  RS_CUDA(cudaMemcpyAsync(P->ptrs, ptrs.data(), sizeof(void*) * ptrs.size(), cudaMemcpyHostToDevice, st));
  RS_CUDA(cudaStreamSynchronize(st));
  P->work_gen = w.gen;
  return RS_OK;
}

// Tile list and counters for (precision, R, tile); built once per handle.
static int get_plan(Handle* h, int prec, int R, int tile, cudaStream_t st, PersPlan** out) {
  if (!h->pers) h->pers = new PersCache();
  PersCache* c = (PersCache*)h->pers;
  RS_TRY(ensure_work_pub(h, prec, R, st));
  for (PersPlan* P : c->plans)
    if (P->prec == prec && P->R == R && (P->TN ? P->TM * 1000 + P->TN : 0) == tile) {
      if (P->work_gen != h->work[prec].gen) RS_TRY(refresh_ptrs(h, P, st));
      *out = P;
      return RS_OK;
    }
  PersPlan* P = new PersPlan();
  c->plans.push_back(P);
  P->prec = prec;
  P->R = R;
  P->CT = ct_for(h->cplx, prec, R);
  P->TN = tile % 1000;
  P->TM = tile ? tile / 1000 : 32;
  const int L = h->L;
  // global box numbering: depth L first, ..., depth 0 last
  std::vector<int> gbase(L + 1);
  int G = 0;
  for (int d = L; d >= 0; --d) { gbase[d] = G; G += h->lv[d].nbox; }
  P->nbox = G;
  std::vector<int> depth(G), n(G), k(G), parent(G), up_need(G, 0), dn_need(G, 0);
  std::vector<int64_t> off(G), skoff(G), uoff(G), loff(G);
  for (int d = 0; d <= L; ++d) {
    const Level& lv = h->lv[d];
    for (int b = 0; b < lv.nbox; ++b) {
      int g = gbase[d] + b;
      depth[g] = d;
      n[g] = lv.h_n[b];
      k[g] = lv.h_k[b];
      off[g] = lv.h_off[b];
      skoff[g] = d > 0 ? lv.h_skoff[b] : 0;
      uoff[g] = lv.h_uoff[b];
      loff[g] = d > 0 ? lv.h_loff[b] : 0;
      parent[g] = d > 0 ? gbase[d - 1] + lv.h_parent[b] : -1;
    }
  }
  // Column ranges per depth: a depth with few row tiles splits its columns
  // (in CT-aligned ranges) so that its tiles still fill the GPU.
  const int nchunk = div_up(R, P->CT);
  const int rb = P->TN ? P->TM : 32;   // rows per tile
  auto col_ranges = [&](int d, bool down) {
    const Level& lv = h->lv[d];
    int64_t rt = 0;
    for (int b = 0; b < lv.nbox; ++b) rt += div_up(down ? lv.h_n[b] : lv.h_n[b] + lv.h_k[b], rb);
    int split = (int)std::max<int64_t>(1, std::min<int64_t>(nchunk, 8192 / std::max<int64_t>(1, rt)));
    int per = div_up(nchunk, split) * P->CT;
    if (P->TN) {   // CTA tiles: whole column blocks, split only while a level has few row tiles
      const int nb = div_up(R, P->TN);
      const int sp = (int)std::max<int64_t>(1, std::min<int64_t>(nb, 2048 / std::max<int64_t>(1, rt)));
      per = div_up(nb, sp) * P->TN;
    }
    std::vector<std::pair<int, int>> cr;
    for (int c = 0; c < R; c += per) cr.push_back({c, std::min(R, c + per)});
    return cr;
  };
  std::vector<Tile> tiles;
  for (int d = L; d >= 1; --d) {
    auto cr = col_ranges(d, false);
    for (int b = 0; b < h->lv[d].nbox; ++b) {
      int g = gbase[d] + b;
      for (int r0 = 0; r0 < n[g] + k[g]; r0 += rb)
        for (auto& c : cr) tiles.push_back(Tile{g, r0, c.first, c.second, T_UP});
      up_need[parent[g]] += div_up(n[g] + k[g], rb) * (int)cr.size();
    }
  }
  {
    auto cr = col_ranges(0, false);
    int g = gbase[0];
    for (int r0 = 0; r0 < n[g]; r0 += rb)
      for (auto& c : cr) tiles.push_back(Tile{g, r0, c.first, c.second, T_ROOT});
    dn_need[g] = div_up(n[g], rb) * (int)cr.size();
  }
  for (int d = 1; d <= L; ++d) {
    auto cr = col_ranges(d, true);
    for (int b = 0; b < h->lv[d].nbox; ++b) {
      int g = gbase[d] + b;
      for (int r0 = 0; r0 < n[g]; r0 += rb)
        for (auto& c : cr) tiles.push_back(Tile{g, r0, c.first, c.second, T_DOWN});
      dn_need[g] = div_up(n[g], rb) * (int)cr.size();
    }
  }
  P->ntiles = (int)tiles.size();
  P->h_tiles = tiles;
  P->h_depth = depth;
  std::vector<int64_t> ldv(L + 1);
  for (int d = 0; d <= L; ++d) ldv[d] = std::max<int64_t>(1, h->lv[d].ntot);
  // every table in one device block and one copy (the plan is built on the
  // first solve of a new handle, where many small allocations and copies
  // would cost more than the solve's own launches)
  HostPack pk;
  const size_t o_tiles = pk.add(tiles), o_depth = pk.add(depth), o_n = pk.add(n), o_k = pk.add(k),
               o_off = pk.add(off), o_skoff = pk.add(skoff), o_uoff = pk.add(uoff), o_loff = pk.add(loff),
               o_parent = pk.add(parent), o_up = pk.add(up_need), o_dn = pk.add(dn_need), o_ldv = pk.add(ldv);
  unsigned char* blk = nullptr;
  RS_TRY(dev_upload(P, &blk, pk.buf, st));
  P->tiles = reinterpret_cast<Tile*>(blk + o_tiles);
  P->bt.depth = reinterpret_cast<int*>(blk + o_depth);
  P->bt.n = reinterpret_cast<int*>(blk + o_n);
  P->bt.k = reinterpret_cast<int*>(blk + o_k);
  P->bt.off = reinterpret_cast<int64_t*>(blk + o_off);
  P->bt.skoff = reinterpret_cast<int64_t*>(blk + o_skoff);
  P->bt.uoff = reinterpret_cast<int64_t*>(blk + o_uoff);
  P->bt.loff = reinterpret_cast<int64_t*>(blk + o_loff);
  P->bt.parent = reinterpret_cast<int*>(blk + o_parent);
  P->bt.up_need = reinterpret_cast<int*>(blk + o_up);
  P->bt.dn_need = reinterpret_cast<int*>(blk + o_dn);
  P->ldv = reinterpret_cast<int64_t*>(blk + o_ldv);
  std::vector<int> zeros(2 + 2 * (size_t)G, 0);
  RS_TRY(dev_upload(P, &P->counters, zeros, st));
  RS_TRY(refresh_ptrs(h, P, st));
  RS_TRY(flag_take(&P->flag_host, &P->flag_dev));
  RS_CUDA(cudaStreamSynchronize(st));
  *out = P;
  return RS_OK;
}

template <class S, class SIO>
static int launch_plan(Handle* h, PersPlan* P, const SIO* B, int64_t ldb, int R, SIO* X, int64_t ldx,
                       const SIO* sub, cudaStream_t st) {
  const int tile = P->TN ? P->TM * 1000 + P->TN : 0;
  switch (tile) {
    case 32032: RS_TRY((launch_pers<S, SIO, 1, 32, 32>(h, P, B, ldb, R, X, ldx, sub, st))); break;
    case 32064: RS_TRY((launch_pers<S, SIO, 1, 32, 64>(h, P, B, ldb, R, X, ldx, sub, st))); break;
    case 64032: RS_TRY((launch_pers<S, SIO, 1, 64, 32>(h, P, B, ldb, R, X, ldx, sub, st))); break;
    case 64064: RS_TRY((launch_pers<S, SIO, 1, 64, 64>(h, P, B, ldb, R, X, ldx, sub, st))); break;
    case 0:
      switch (P->CT) {
        case 1: RS_TRY((launch_pers<S, SIO, 1, 32, 0>(h, P, B, ldb, R, X, ldx, sub, st))); break;
        case 8: RS_TRY((launch_pers<S, SIO, 8, 32, 0>(h, P, B, ldb, R, X, ldx, sub, st))); break;
        case 16: RS_TRY((launch_pers<S, SIO, 16, 32, 0>(h, P, B, ldb, R, X, ldx, sub, st))); break;
        case 32: RS_TRY((launch_pers<S, SIO, 32, 32, 0>(h, P, B, ldb, R, X, ldx, sub, st))); break;
        default: return fail(RS_ERR_ARG, "bad column tile");
      }
      break;
    default: return fail(RS_ERR_ARG, "bad column tile");
  }
  h->pers_last = P;
  return RS_OK;
}

template <class S, class SIO>
static int pers_impl(Handle* h, int prec, const SIO* B, int64_t ldb, int R, SIO* X, int64_t ldx, cudaStream_t st,
                     const SIO* sub = nullptr) {
  int bucket = 1;
  while (bucket * 2 <= R) bucket *= 2;
  const TuneKey key{prec, bucket, h->cplx ? 1 : 0, h->N};
  int known = -1;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) known = it->second;
  }
  const bool tc = TcOk<S, SIO>::value && tc_enabled() && R <= TC_MAX_COLS && tc_shallow(h);
  const std::vector<int> cand = launch_configs(R, tc);
  PersPlan* P = nullptr;
  // one launch of configuration cfg (tile * 16 + CTAs per SM): tensor-core
  // tiles go to solve_tc.cu, the others to the persistent kernels here
  auto run = [&](int cfg) -> int {
    const int tile = cfg / 16;
    if (tile / 1000 == TC_TM) {
      if constexpr (TcOk<S, SIO>::value)
        return solve_tc_run(h, prec, tile % 1000, (const double*)B, ldb, R, (double*)X, ldx, (const double*)sub, st);
      return fail(RS_ERR_ARG, "solve: tensor-core tiles need float arithmetic on real kernels");
    }
    RS_TRY(get_plan(h, prec, R, tile, st, &P));
    P->cps = cfg % 16;
    tc_forget_last(h);
    return launch_plan<S, SIO>(h, P, B, ldb, R, X, ldx, sub, st);
  };
  {   // an override (rs_set_path "tile:...") replaces the tuned choice
    int f = solve_tile_force();
    if (f >= 0) {
      if (R < 16 || (f / 1000 == TC_TM && !(TcOk<S, SIO>::value && R <= TC_MAX_COLS && tc_shallow(h))))
        f = f == 0 || R < 16 ? 0 : 32064;
      return run(f * 16);
    }
  }
  // Repeating the launch is only harmless when the output overwrites neither
  // input (in-place solves and the in-place residual update are not tuned;
  // the update borrows the FP32 solve's choice).
  const bool aliased = (const void*)X == (const void*)B || (sub && (const void*)X == (const void*)sub);
  if (known < 0 && aliased && prec == MODE_FWD_F32) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(TuneKey{RS_PREC_FP32, bucket, key.cplx, key.N});
    if (it != g_tuned.end()) known = it->second;
  }
  if (known >= 0 && (known / 16) / 1000 == TC_TM && !tc) known = -1;   // not available here
  if (known >= 0 || cand.size() == 1 || aliased) return run(known >= 0 ? known : cand[0]);
  // autotune: time the second of two launches of each candidate (the first
  // pays one-time costs); the outputs agree bit for bit
  cudaEvent_t e0, e1;
  RS_CUDA(cudaEventCreate(&e0));
  RS_CUDA(cudaEventCreate(&e1));
  int best = cand[0];
  float best_ms = 1e30f;
  int rc = RS_OK;
  for (int cfg : cand) {
    if ((rc = run(cfg)) != RS_OK) break;
    cudaEventRecord(e0, st);
    if ((rc = run(cfg)) != RS_OK) break;
    cudaEventRecord(e1, st);
    float ms = 0;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaGetLastError();
      rc = fail(RS_ERR_CUDA, "solve: autotuning timing failed");
      break;
    }
    if (ms < best_ms) {
      best_ms = ms;
      best = cfg;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == RS_OK) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = best;
  }
  // the candidates do not all round alike (tensor-core and CUDA-core tiles):
  // leave the chosen configuration's result in X
  if (rc == RS_OK && best != cand.back()) rc = run(best);
  return rc;
}

int solve_pers_device(Handle* h, int prec, const void* d_B, int64_t ldb, int nrhs, void* d_X, int64_t ldx,
                      cudaStream_t st) {
  if (h->cplx) {
    if (prec == RS_PREC_FP64) return pers_impl<c128, c128>(h, prec, (const c128*)d_B, ldb, nrhs, (c128*)d_X, ldx, st);
    return pers_impl<c64, c128>(h, prec, (const c128*)d_B, ldb, nrhs, (c128*)d_X, ldx, st);
  }
  if (prec == RS_PREC_FP64) return pers_impl<double, double>(h, prec, (const double*)d_B, ldb, nrhs, (double*)d_X, ldx, st);
  return pers_impl<float, double>(h, prec, (const double*)d_B, ldb, nrhs, (double*)d_X, ldx, st);
}

int solve_pers_device_sub(Handle* h, int mode, const double* d_B, int64_t ldb, int nrhs, double* d_X, int64_t ldx,
                          const double* d_sub, cudaStream_t st) {
  if (mode != MODE_FWD_F32 && mode != MODE_FWD_DF) return fail(RS_ERR_ARG, "forward operator: bad mode");
  if (h->cplx) {   // the buffers hold complex double values
    const c128 *B = (const c128*)d_B, *sub = (const c128*)d_sub;
    if (mode == MODE_FWD_DF) return pers_impl<cdfloat, c128>(h, mode, B, ldb, nrhs, (c128*)d_X, ldx, st, sub);
    return pers_impl<c64, c128>(h, mode, B, ldb, nrhs, (c128*)d_X, ldx, st, sub);
  }
  if (mode == MODE_FWD_DF) return pers_impl<dfloat, double>(h, mode, d_B, ldb, nrhs, d_X, ldx, st, d_sub);
  return pers_impl<float, double>(h, mode, d_B, ldb, nrhs, d_X, ldx, st, d_sub);
}

// After the stream has been synchronized: timeout flags of every plan that
// ran since the last check.
// Tile timeline of the last profiled persistent launch of plan (prec, R):
// per tile its kind, depth, rows from, columns, and the times (us, from the
// earliest claim) it was claimed, its dependencies were met and it finished.
int tile_trace(Handle* h, int prec, int R, int64_t cap, int* kind, int* depth, int* r0, int* ncol, double* t_claim,
               double* t_start, double* t_end, int64_t* count) {
  if (tc_tile_trace(h, prec, R, cap, kind, depth, r0, ncol, t_claim, t_start, t_end, count) == RS_OK) return RS_OK;
  PersCache* c = (PersCache*)h->pers;
  PersPlan* P = nullptr;
  if (c)
    for (PersPlan* q : c->plans)
      if (q->prec == prec && q->R == R && q->traced) P = q;
  PersPlan* last = (PersPlan*)h->pers_last;
  if (last && last->prec == prec && last->R == R && last->traced) P = last;
  if (!P) return fail(RS_ERR_STATE, "rs_profile_tiles: no profiled launch of this plan");
  std::vector<unsigned long long> tr(3 * (size_t)P->ntiles);
  RS_CUDA(cudaDeviceSynchronize());
  RS_CUDA(cudaMemcpy(tr.data(), P->trace, sizeof(unsigned long long) * tr.size(), cudaMemcpyDeviceToHost));
  unsigned long long t0 = ~0ull;
  for (int t = 0; t < P->ntiles; ++t) t0 = std::min(t0, tr[3 * (size_t)t]);
  const int64_t n = std::min<int64_t>(cap, P->ntiles);
  for (int64_t t = 0; t < n; ++t) {
    const Tile& tl = P->h_tiles[t];
    if (kind) kind[t] = tl.kind;
    if (depth) depth[t] = P->h_depth[tl.g];
    if (r0) r0[t] = tl.r0;
    if (ncol) ncol[t] = tl.c1 - tl.c0;
    if (t_claim) t_claim[t] = 1e-3 * (double)(tr[3 * t] - t0);
    if (t_start) t_start[t] = 1e-3 * (double)(tr[3 * t + 1] - t0);
    if (t_end) t_end[t] = 1e-3 * (double)(tr[3 * t + 2] - t0);
  }
  if (count) *count = P->ntiles;
  return RS_OK;
}

int pers_check(Handle* h) {
  RS_TRY(tc_check(h));
  PersCache* c = (PersCache*)h->pers;
  if (!c) return RS_OK;
  int rc = RS_OK;
  for (PersPlan* P : c->plans)
    if (P->flag_host && *(volatile int*)P->flag_host) {
      P->dirty = true;
      *P->flag_host = 0;
      rc = RS_ERR_TIMEOUT;
    }
  if (rc != RS_OK) return fail(RS_ERR_TIMEOUT, "solve: a dependency wait ran out (flag set by the device)");
  return RS_OK;
}

}  // namespace rs
