// Internal runtime structures of the recursive-skeletonization library.
//
// Device data layout (one handle):
//   pts      coordinates per axis in tree order (x, y[, z]), N doubles each
//   perm     tree position -> caller's point index
//   per tree depth d = 0..L (Level):
//     box tables from the tree (begin, parent, child range, colleagues)
//     active set of each box: ids of points (tree positions) in `act`,
//       box b at act[off[b] .. off[b] + n[b]); at the leaves act = identity;
//       above, the concatenated skeletons of the children (child order)
//     owner[pos]: the child box (depth d+1) a position of depth d came from
//     ID output: k[b], lperm (per box a permutation of 0..n-1: first k =
//       skeletons in pivot order, then the redundant ones), T (k x (n-k)
//       column-major at toff[b])
//     skoff[b]: where box b's skeletons start in the depth d-1 active vector
//     factors (eq. compressed-inverse), column-major:
//       U   at uoff[b]: (n+k) x n = [calD ; calR]
//       Lf  at loff[b]: n x k     = calL
//       Lam at lamoff[b]: k x k   = Lambda (read by the parent's assembly)
//     float copies U32 / Lf32 for the mixed-precision solve
//     forward factors FU32/FUdf ((n+k) x n = [D ; P] at uoff) and FL32/FLdf
//       (n x k = P^T at loff): float and double-float (real kernels),
//       complex float and complex double-float (complex kernels)
//   the root is depth 0 with k = 0, so its U holds calS^{-1}.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "rs_common.cuh"

namespace rs {

// ------------------------------------------------------------- profiler
enum ProfCat { P_TREE, P_ID, P_FACTOR, P_COPY32, P_UP, P_DOWN, P_PERM, P_FWD_PROJ, P_FWD_DBLOCK, P_FWD_DOWN,
               P_RESID, P_MISC, P_SOLVE64, P_SOLVE32, P_NCAT };
bool prof_on();
bool prof_tiles_on();   // rs_profile_enable(2): tile timelines as well
void prof_begin(int cat, cudaStream_t st);
void prof_end(int cat, cudaStream_t st, double bytes, double flops);
void prof_amend(int cat, double bytes, double flops);  // fix up the last record of cat

// ------------------------------------------------------------ primitives
// Exclusive scan of n int64 values; *total (host) receives the sum.
int scan_i64(const int64_t* d_in, int64_t* d_out, int64_t n, int64_t* total, cudaStream_t st);
// Exclusive scan of int32 values into int64 offsets.
int scan_i32_to_i64(const int* d_in, int64_t* d_out, int64_t n, int64_t* total, cudaStream_t st);
// Stable LSD radix sort of (key, value) pairs on the low `bits` key bits.
int radix_sort_pairs(uint64_t* keys, int* vals, uint64_t* keys_tmp, int* vals_tmp, int n, int bits,
                     cudaStream_t st);
// Max / sum of an int array (host result).
int reduce_max_i32(const int* d_in, int n, int* out, cudaStream_t st);

// Device buffer owned by a handle.
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Level {
  int depth = 0;
  int nbox = 0;
  // tree
  int* begin = nullptr;        // first point (tree order) of each box
  int* parent = nullptr;       // parent box at depth-1
  int* child_begin = nullptr;  // children at depth+1 are [child_begin, child_end)
  int* child_end = nullptr;
  int* ncoll = nullptr;
  int* coll = nullptr;         // 27 per box, ascending, -1 padded
  int* coords = nullptr;       // dim per box
  uint64_t* keys = nullptr;
  // active sets
  int64_t ntot = 0;            // sum of n over boxes
  int* n = nullptr;
  int64_t* off = nullptr;
  int* act = nullptr;
  int* owner = nullptr;        // child box of each active position (depth < L)
  // skeletonization
  int* k = nullptr;
  int64_t* skoff = nullptr;
  int* lperm = nullptr;        // ntot entries
  int64_t* toff = nullptr;
  int64_t* uoff = nullptr;
  int64_t* loff = nullptr;
  int64_t* lamoff = nullptr;
  void* T = nullptr;
  void* U = nullptr;
  void* Lf = nullptr;
  void* Lam = nullptr;
  void* U32 = nullptr;
  void* Lf32 = nullptr;
  // forward operator in the solve's two-pass form (fwd2.cu): FU = [D ; P]
  // ((n+k) x n at uoff) and FL = P^T (n x k at loff), low and high precision
  void* FU32 = nullptr;
  void* FL32 = nullptr;
  void* FUdf = nullptr;
  void* FLdf = nullptr;
  // row side of a non-symmetric kernel (row active set, row ID's column
  // order and T, at the same offsets as the column side); for symmetric
  // kernels these alias act, lperm and T
  int* act_r = nullptr;
  int* lperm_r = nullptr;
  void* T_r = nullptr;
  int64_t ksum = 0;            // sum of k (size of depth-1 active vector)
  int64_t usz = 0, lsz = 0, lamsz = 0, tsz = 0;  // scalars in the pools
  int maxn = 0, maxm = 0, maxk = 0;
  // host copies (for sizes and the inspection API)
  std::vector<int> h_n, h_k, h_begin, h_parent, h_ncoll, h_coll;
  std::vector<int64_t> h_off, h_skoff, h_uoff, h_loff;
};

struct Handle {
  int device = -1;             // CUDA device the handle was built on (its memory lives there)
  int dim = 2;
  int64_t N = 0;
  KParams kp{};
  int nproxy = 64;
  double ratio = 1.5;
  double eps = 1e-9;
  int leaf = 64;
  bool cplx = false;
  bool id_df = false;          // double-float pivoted QR in the ID (real kernels)
  int id_p = 0;                // randomized ID: oversampling rows of the sample (0: deterministic CPQR)
  uint64_t id_seed = 0;        // seed of the sample's normal stream
  double* sketch = nullptr;    // sketch table (SKETCH_STRIDE x sketch_m), from the handle's memory
  int sketch_m = 0;
  int L = 0;
  double center[3] = {0, 0, 0};
  double half = 1.0;           // root half-width a
  double* pts = nullptr;       // 3 * N (x, y, z blocks)
  double* dlg = nullptr;       // double layer: 3 * N (normal x, normal y, curvature), tree order
  bool nonsym = false;         // non-symmetric kernel: two-sided IDs
  int* perm = nullptr;
  std::vector<Level> lv;       // index = depth
  std::vector<void*> allocs;   // pool blocks owned by the handle (freed by rs_free)
  cudaStream_t bst = nullptr;  // stream of the build (allocations are ordered on it)
  cudaStream_t fst = nullptr;  // during the build: the factorization stream, which runs
                               // behind the skeletonization on bst
  cudaEvent_t aev = nullptr;   // orders fst after a new device block taken on bst
  char* arena_cur = nullptr;   // bump pointer into the current block
  size_t arena_left = 0;
  double build_ms = 0;
  int64_t factor_scalars = 0;
  int* status = nullptr;       // device status word (singularity etc.)
  // solve workspaces (grown on demand)
  struct Work {
    int R = 0;
    int prec = -1;
    void* vin = nullptr;        // caller-order staging (double / c128), N*R
    std::vector<void*> v;       // per depth: input vector of the upward pass
    std::vector<void*> u;       // per depth: calD b, then x in the downward pass
    size_t bytes = 0;
    int gen = 0;                // bumped whenever the buffers are reallocated
  };
  Work work[4];                 // [0] FP64 solve, [1] FP32 solve, [2] float forward, [3] double-float forward
  // refinement / matvec workspaces
  void* r64 = nullptr; void* x64 = nullptr; void* b64 = nullptr;
  std::vector<void*> fz, fy;    // forward operator vectors per depth
  int fR = 0;
  double* colnorm = nullptr;    // 2 * R
  int ncolnorm = 0;
  void* pers = nullptr;         // persistent-solve plans (solve2.cu)
  void* pers_tc = nullptr;      // tensor-core solve plans (solve_tc.cu)
  void* pers_last = nullptr;
};

// fault injection (api.cu): true once after rs_set_fault("wait")
bool take_wait_fault();

// Build-path selection override (rs_set_path, for tests that reach the
// multi-CTA fallbacks on small problems) and per-path launch counters
// (rs_path_counts).  The override only removes choices: every path it
// leaves is one the production selection can take.
enum PathForce {
  PF_ID_BIG = 1,          // every ID level on the multi-CTA path (run_id_big)
  PF_ID_NOCLUSTER = 2,    // ... without the thread-block-cluster form
  PF_ID_NOCOOP = 4,       // ... and without the cooperative form (one launch per pivot step)
  PF_FACTOR_BIG = 8,      // every factorization level on the multi-CTA path
  PF_GJ_NOCLUSTER = 16,   // Gauss-Jordan steps without the cluster form
  PF_GJ_NOBLOCKED = 32,   // ... without the blocked form
  PF_GJ_NOCOOP = 64       // ... without the cooperative form
};
enum PathId {
  PATH_ID_CTA, PATH_ID_CLUSTER, PATH_ID_COOP, PATH_ID_STEP,
  PATH_FAC_SMEM, PATH_FAC_BIG, PATH_FAC_GENERIC,
  PATH_GJ_CLUSTER, PATH_GJ_BLOCKED, PATH_GJ_COOP, PATH_GJ_STEP, PATH_N
};
int path_force();
void path_count(int which);
// Solve tile override (rs_set_path "tile:..."): -1 = the autotuner's choice,
// 0 = the warp kernel, else TM * 1000 + TN.
int solve_tile_force();

// Mapped pinned int flags (a persistent launch's error flag, read by the
// host after the launch) from a process-wide pool: one cudaHostAlloc costs
// more than the rest of a solve plan's set-up, and every new handle builds
// plans.  flag_take gives a zeroed flag's host and device addresses;
// flag_release returns it to the pool.
int flag_take(int** host, int** dev);
void flag_release(int* host);

// Several small host tables staged for one device allocation and one copy.
struct HostPack {
  std::vector<unsigned char> buf;
  size_t add_bytes(const void* p, size_t bytes);
  template <class T> size_t add(const std::vector<T>& v) { return add_bytes(v.data(), sizeof(T) * v.size()); }
};

// allocation helper: records in h->allocs
int dalloc(Handle* h, void** p, size_t bytes);
template <class T> int dalloc_t(Handle* h, T** p, size_t count) {
  return dalloc(h, (void**)p, count * sizeof(T));
}

// Tree construction (tree.cu).
int build_tree(Handle* h, const double* d_pts_in, cudaStream_t st);

// Skeletonization + factorization of one depth (skel.cu).
// The skeletonization of a depth runs on st; its factorization is queued on
// fs behind it (fs waits for the depth's ID on st and runs the depths in
// order), so the IDs of the next depths overlap the factorizations.
int skeletonize_level(Handle* h, int depth, cudaStream_t st, cudaStream_t fs);
int factor_root(Handle* h, cudaStream_t st, cudaStream_t fs);
// After fs has been joined into st: the factorizations' status words.
int check_factor_status(Handle* h, cudaStream_t st);
int make_fp32_copies(Handle* h, cudaStream_t st);

// Solve / forward operator (solve.cu).
int solve_device(Handle* h, int prec, const void* d_B, int64_t ldb, int nrhs, void* d_X, int64_t ldx,
                 cudaStream_t st);
int matvec_device(Handle* h, const void* d_X, int64_t ldx, int nrhs, void* d_Y, int64_t ldy,
                  cudaStream_t st);
int colnorm2_device(Handle* h, const void* d_v, int nrhs, double* d_out, cudaStream_t st);
int axpy_lowp_device(Handle* h, void* d_x, const void* d_d, int nrhs, cudaStream_t st);
// Forward operator of the refinement from the stored forward factors (fwd2.cu).
int make_fwd_blocks(Handle* h, cudaStream_t st);
int residual_df(Handle* h, const double* b, const double* x, double* r, int R, bool full, cudaStream_t st);

// Persistent single-launch solve (solve2.cu).  Besides RS_PREC_FP64 and
// RS_PREC_FP32 it runs the forward operator from the forward factors and
// then writes X = sub - A_RS B: MODE_FWD_F32 in float (complex float),
// MODE_FWD_DF in double-float (complex double-float).
enum { MODE_FWD_F32 = 2, MODE_FWD_DF = 3 };
int solve_pers_device_sub(Handle* h, int mode, const double* d_B, int64_t ldb, int nrhs, double* d_X, int64_t ldx,
                          const double* d_sub, cudaStream_t st);
int solve_pers_device(Handle* h, int prec, const void* d_B, int64_t ldb, int nrhs, void* d_X, int64_t ldx,
                      cudaStream_t st);
int pers_check(Handle* h);
// Tensor-core multi-column solve (solve_tc.cu): mode RS_PREC_FP32 or
// MODE_FWD_F32 on real kernels, TN in {64, 128, 256} columns per unit, at
// most TC_MAX_COLS columns per call.
constexpr int TC_MAX_COLS = 1024;
int solve_tc_run(Handle* h, int mode, int TN, const double* B, int64_t ldb, int R, double* X, int64_t ldx,
                 const double* sub, cudaStream_t st);
int tc_check(Handle* h);
int tc_tile_trace(Handle* h, int mode, int R, int64_t cap, int* kind, int* depth, int* r0, int* ncol,
                  double* t_claim, double* t_start, double* t_end, int64_t* count);
void tc_forget_last(Handle* h);
void free_tc(Handle* h);
int tile_trace(Handle* h, int prec, int R, int64_t cap, int* kind, int* depth, int* r0, int* ncol, double* t_claim,
               double* t_start, double* t_end, int64_t* count);
void free_pers(Handle* h);
int prec_cat(int prec);
int ensure_work_pub(Handle* h, int prec, int R, cudaStream_t st);
// Block-diagonal preconditioned GMRES over several patches (gmres.cu); d_pts
// per axis (x[n], y[n], z[n]) in the caller's order, b and x device vectors.
int gmres_patches_device(int np, Handle* const* hs, const double* d_pts, const void* b, void* x, double tol,
                         int max_it, int restart, int precondition, int* its_out, double* relres_out,
                         cudaStream_t st);
// Solve with the per-level vectors in the library's static device scratch.
int solve_noalloc_device(Handle* h, int prec, const void* d_B, int64_t ldb, int nrhs, void* d_X, int64_t ldx,
                         cudaStream_t st);

}  // namespace rs
