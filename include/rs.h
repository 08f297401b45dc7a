/*
 * rs.h -- C ABI of the GB300 recursive-skeletonization fast direct solver.
 *
 * The library builds a compressed inverse of a dense matrix A = I + w K,
 * K_ij = G(x_i, x_j) (i != j), K_ii = 0, for points x_1..x_N on a curve or
 * surface, following Ho & Greengard, "A fast direct solver for structured
 * linear systems by recursive skeletonization" (arXiv 1110.3105):
 *   - tree: uniform quadtree / octree with contiguous index blocks
 *     (Sec. 2.1, Example 1; Sec. 6, first paragraph);
 *   - compression: interpolative decomposition (Sec. 2.2, Def. 2.3) of each
 *     box against its near neighbours and a proxy surface (Sec. 3.1-3.2),
 *     level by level (eq. multilevel-compression);
 *   - factorization: block elimination of the sparse embedding
 *     (eq. compressed-inverse, eq. multilevel-inverse, Sec. 3.4);
 *   - solve: the telescoping inverse applied level by level (Sec. 4.3).
 * Green's functions: eq. 2d-laplace, eq. 3d-laplace, eq. 2d-helmholtz,
 * eq. 3d-helmholtz, and the 2D double-layer kernel of eq. double-layer
 * (non-symmetric: separate row and column skeletons, Sec. 3.1).
 *
 * Conventions (all entry points):
 *   - Return value: RS_OK (0) or a negative RS_ERR_* code.  On error no
 *     output handle is created and rs_last_error() gives a message for the
 *     calling thread (valid until its next library call).
 *   - Pointers may be host or device memory; the library detects which.
 *     The caller owns every buffer it passes; the library copies what it
 *     keeps.  A handle owns all device memory it allocates until rs_free.
 *   - Vectors are N x nrhs, column-major with leading dimension ld >= N, in
 *     the caller's original point order.  Real kernels use double, the
 *     Helmholtz kernels interleaved double complex (re, im).
 *   - stream: a cudaStream_t (NULL = legacy default stream).  Calls are
 *     stream-ordered; a call returns after its results are complete and, for
 *     host outputs, copied back.
 *   - A handle is not thread-safe: calls on one handle must be serialised.
 *   - Everything runs on the current CUDA device.
 */
#ifndef RS_H_
#define RS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum rs_status {
  RS_OK = 0,
  RS_ERR_ARG = -1,      /* invalid argument */
  RS_ERR_OOM = -2,      /* device or host allocation failed */
  RS_ERR_CUDA = -3,     /* CUDA runtime error */
  RS_ERR_SINGULAR = -4, /* a diagonal block or Lambda was numerically singular */
  RS_ERR_TIMEOUT = -5,  /* a bounded wait ran out */
  RS_ERR_NAN = -6,      /* non-finite input or result */
  RS_ERR_STATE = -7     /* call not valid in the handle's current state */
};

enum rs_kernel {
  RS_LAPLACE2D = 0,   /* G = -(1/2 pi) log r          (eq. 2d-laplace)   */
  RS_HELMHOLTZ2D = 1, /* G = (i/4) H0^(1)(k r)         (eq. 2d-helmholtz) */
  RS_LAPLACE3D = 2,   /* G = 1 / (4 pi r)              (eq. 3d-laplace)   */
  RS_HELMHOLTZ3D = 3, /* G = e^{i k r} / (4 pi r)      (eq. 3d-helmholtz) */
  RS_LAPLACE2D_DL = 4 /* K = dG/dnu_y = (1/2 pi) (x - y).nu_y / r^2, the 2D
                         double layer (eq. double-layer, Sec. 6.2); needs
                         rs_params.normals and .curvature; K_ii = -kappa_i/(4 pi) */
};

enum rs_precision {
  RS_PREC_FP64 = 0,   /* stored factors and arithmetic in double (complex double) */
  RS_PREC_FP32 = 1    /* float (complex float) copies of the factors */
};

typedef struct rs_handle_s* rs_handle;

/* Build parameters.  proxy_n: points on the proxy surface (2D: a circle of
 * radius proxy_ratio * box circumradius; 3D: 6 g^2 cell centres on a cube of
 * half-width proxy_ratio * box half-width, Sec. 3.2).  weight: w in A. */
/* Arithmetic of the ID's pivoted QR (Sec. 2.2) for real kernels.  RS_ID_FP64
 * (0, the default) runs it in FP64.  RS_ID_DFLOAT runs the O(m n) passes in
 * double-float arithmetic on the FP32 pipes (hi + lo floats, ~48 significant
 * bits; backward error ~1e-12, far below any eps >= 1e-10), with the norms,
 * R_jj and the stopping test still in FP64 scalars; ranks then agree with the
 * FP64 build up to pivot near-ties.  Complex kernels always use FP64. */
enum rs_id_arith {
  RS_ID_FP64 = 0,
  RS_ID_DFLOAT = 1
};

/* Randomized ID (Sec. 2.2: the paper's ID compresses a random sample of a
 * box's matrix instead of the matrix).  With id_oversample = p > 0, a box
 * whose compressed matrix M (m x n) has m > n + p is compressed through the
 * sample Omega M of n + p rows (the same pivoted QR and rank rule), Omega
 * having independent N(0,1) entries: entry (i, r) is element r * 1024 + i of
 * the normal stream 77 of id_seed (splitmix64 counters, Box-Muller pairs),
 * the same numbers the package's input module draws.  Boxes compressed by
 * the multi-CTA forms (too large for one CTA) are sampled the same way.
 * Needs id_arith = RS_ID_FP64 and every box's n + p <= 1024; p = 0 keeps the
 * deterministic ID.  The paper samples with a structured random transform;
 * the Gaussian sample is the plain form of the same scheme. */
/* Non-symmetric kernels (RS_LAPLACE2D_DL).  Every box gets a column ID of
 * its off-diagonal block column (outgoing skeletons; proxy rows: the kernel
 * at the proxy points as targets) and a row ID of its off-diagonal block row
 * (incoming skeletons; proxy rows: single-layer charges on the proxy circle
 * and a constant as sources), both at the rank max(row rank, column rank)
 * (Sec. 3.1, in the equal-dimension form of Sec. 3.4's block elimination).
 * The second-kind equation -sigma/2 + D sigma = f of eq. 2k-integral-eqn is
 * A sigma = -2 f with weight w = -2 h.  normals: 2 x N column-major outward
 * unit normals (point i at normals[2 i], normals[2 i + 1]); curvature: N
 * values; both host or device, in the caller's point order, copied at build;
 * ignored (may be NULL) for the other kernels.  These builds take the
 * one-CTA-per-box ID and the general block elimination; the randomized ID
 * and the double-float ID are not available for them. */
typedef struct {
  int kernel_id;      /* enum rs_kernel */
  double k_wave;      /* Helmholtz wavenumber k > 0 (ignored otherwise) */
  double weight;      /* w: > 0, or any finite nonzero value for RS_LAPLACE2D_DL */
  int proxy_n;        /* > 0; 3D needs 6 g^2 */
  double proxy_ratio; /* > 1 */
  int id_arith;       /* enum rs_id_arith */
  int id_oversample;  /* randomized ID oversampling p (0: deterministic CPQR), 0..512 */
  uint64_t id_seed;   /* seed of the randomized ID's sample */
  const double* normals;    /* RS_LAPLACE2D_DL: 2 x N outward unit normals */
  const double* curvature;  /* RS_LAPLACE2D_DL: N curvatures */
} rs_params;

/* Summary of a built handle (Table solve-lap-2d fields plus timings). */
typedef struct {
  int64_t n;              /* matrix dimension N */
  int dim;                /* 2 or 3 */
  int depth;              /* tree depth L (root = 0) */
  int64_t top_skeletons;  /* skeletons left at the root (K at the top) */
  int64_t factor_bytes;   /* FP64 factor storage read by one solve */
  int64_t factor_scalars; /* stored scalars of calD, calL, calR and the root */
  double build_ms;        /* wall time of rs_build on the device timeline */
  int max_box_n;          /* largest active set of any box */
  int max_box_m;          /* largest compressed matrix row count */
  int max_rank;           /* largest skeleton count of any box */
} rs_stats_t;

/* Build the compressed inverse.
 *   pts    dim x N column-major (point i at pts[i*dim .. i*dim+dim-1]), host
 *          or device; N >= 1; dim 3 with RS_LAPLACE3D and RS_HELMHOLTZ3D,
 *          dim 2 with the 2D kernels.  The Helmholtz kernels build and solve
 *          in complex arithmetic (interleaved re, im).
 *   eps    relative ID precision (Sec. 2.2), 0 < eps < 1.
 *   leaf   maximum points per leaf box, >= 1.
 * Errors: RS_ERR_ARG (bad sizes, parameters), RS_ERR_NAN (non-finite point),
 *         RS_ERR_SINGULAR, RS_ERR_OOM, RS_ERR_CUDA. */
int rs_build(const double* pts, int64_t n, int dim, const rs_params* params,
             double eps, int leaf, void* stream, rs_handle* out);

/* X = A_RS^{-1} B (eq. multilevel-inverse), nrhs >= 1, in the given precision.
 * RS_PREC_FP32 takes and returns double data but computes with the float
 * factors.  B and X may alias only if ldb == ldx. */
int rs_solve(rs_handle h, int precision, const void* B, int64_t ldb, int nrhs,
             void* X, int64_t ldx, void* stream);

/* Allocation-free variant of rs_solve (the paper has no counterpart: it is a
 * deployment form).  For callers that cannot allocate device memory during a
 * solve: a latency-critical serving loop (cudaMalloc/cudaFree may synchronize
 * the device and stall other streams' work) or a process whose device-memory
 * budget is fixed at start-up.  Same arguments and result as rs_solve, except:
 *   - B and X must be device memory (RS_ERR_ARG otherwise: host buffers would
 *     need a staging allocation), and the current device must be the one the
 *     handle was built on (RS_ERR_ARG otherwise: the scratch array used is
 *     the current device's);
 *   - the per-level solve vectors live in one static device array of
 *     RS_NOALLOC_SCRATCH_BYTES that every GPU which loads the library holds
 *     until the process exits; a solve needing more (about 2 * nrhs * scalar
 *     size * (N + sum of skeleton counts)) is rejected with RS_ERR_ARG and a
 *     message giving the need and the limit;
 *   - the call allocates nothing (no cudaMalloc/cudaFree, no allocating
 *     library routine).  Its first call on a device looks up the array's
 *     device address (cudaGetSymbolAddress) with that device current; make
 *     that first call before any stream capture;
 *   - every call, on every handle, shares the one array and leaves its last
 *     contents there (nothing in it needs to start at zero): calls whose
 *     work overlaps on the GPU race -- serialise them on one stream. */
#define RS_NOALLOC_SCRATCH_BYTES (16u << 20)
int rs_solve_noalloc(rs_handle h, int precision, const void* B, int64_t ldb, int nrhs,
                     void* X, int64_t ldx, void* stream);

/* Mixed-precision solve with iterative refinement: x0 = FP32 solve of b;
 * r0 = b - A_RS x0 (forward operator of eq. multilevel-compression from its
 * stored blocks, double-float products -- about 48 significant bits; complex
 * kernels: complex double-float); then repeat x += FP32 solve of r and
 * r -= A_RS d (float products on the small correction) until every column
 * has ||r|| <= tol ||b|| or max_it corrections were applied.
 *   its_out     (host, may be NULL) corrections applied
 *   relres_out  (host, may be NULL, nrhs entries) final ||r||/||b|| per column
 * Returns RS_OK even when tol was not met; check relres_out. */
int rs_solve_refined(rs_handle h, const void* B, int64_t ldb, int nrhs, void* X,
                     int64_t ldx, double tol, int max_it, int* its_out,
                     double* relres_out, void* stream);

/* Y = A_RS X in FP64 (Sec. 3.3: upward pass with R^(l), kernel blocks
 * D^(l) and S from the coordinates, downward pass with L^(l)). */
int rs_matvec(rs_handle h, const void* X, int64_t ldx, int nrhs, void* Y,
              int64_t ldy, void* stream);

/* Fill *out with the handle's summary: N, the tree depth, K at the top and
 * the stored-factor size are the quantities the paper's tables list per run
 * (Tables apply-lap-2ds to solve-lap-3d: N, K_row = K_col, M), the build
 * time their T_cm + T_lu; the box maxima have no counterpart in the paper.
 * Errors: RS_ERR_ARG (null handle or output). */
int rs_stats(rs_handle h, rs_stats_t* out);

/* Tree export for bit-exact comparison (host buffers, caller allocated).
 * rs_tree_level(h, l, ...) for l = 0..depth:
 *   nbox_out   number of boxes at depth l
 *   begin      (nbox) first point of each box in tree order, or NULL
 *   parent     (nbox) parent box index at depth l-1 (-1 at the root), or NULL
 *   ncoll      (nbox) colleague count, or NULL
 *   coll       (nbox * 27) colleague box indices ascending, -1 padded, or NULL
 * rs_tree_perm(h, perm): perm[i] = original index of the point at tree
 * position i (int64, N entries).  The tree is the paper's uniform orthtree
 * with contiguous boxes (Sec. 2.1, Example 1).  Errors: RS_ERR_ARG for a
 * null handle, a null perm or a level out of range. */
int rs_tree_perm(rs_handle h, int64_t* perm);
int rs_tree_level(rs_handle h, int level, int* nbox_out, int64_t* begin,
                  int* parent, int* ncoll, int* coll);

/* Per-box ranks at depth l (1..depth): n (active size) and k (skeletons,
 * the ID ranks of Sec. 2.2), host arrays of nbox entries, either may be
 * NULL.  Errors: RS_ERR_ARG for a null handle or a level out of range. */
int rs_box_ranks(rs_handle h, int level, int* n, int* k);

/* Launch profiler (off by default).  rs_profile_enable(1) clears the record
 * and times every following kernel launch of the library with CUDA events
 * on the stream it runs on, grouped into rs_profile_ncat() categories
 * ("tree", "id", "factor", "solve_fp64", "solve_fp32", "residual", ...);
 * rs_profile_enable(2) also records the tile timeline of every persistent
 * solve launch (rs_profile_tiles; a few stores per tile, and the first
 * launch of each plan allocates its buffer); rs_profile_enable(0) stops
 * recording.  rs_profile_read waits for the
 * recorded events and returns, for one category, the summed device time
 * (ms), the launch count and the algorithmic bytes and flops of those
 * launches (counted from the block sizes).  *name is a static string. */
int rs_profile_enable(int on);
int rs_profile_ncat(void);
int rs_profile_read(int cat, double* ms, int64_t* launches, double* bytes, double* flops,
                    const char** name);

/* Individual records of the profiler in launch order: rs_profile_nrec()
 * records; record i gives its category, device time (ms), bytes, flops. */
int rs_profile_nrec(void);
int rs_profile_record(int i, int* cat, double* ms, double* bytes, double* flops);
/* Start of record i in ms after the start of record 0 (gaps between records
 * are host time or launch latency). */
int rs_profile_record_start(int i, double* start_ms);
/* Tile timeline of the last persistent solve launch made while
 * rs_profile_enable(2) was on, for the plan of `mode` (RS_PREC_FP64 or RS_PREC_FP32 solve; 2: float
 * and 3: double-float forward operator of the refinement residual) and nrhs
 * columns.  Each tile is a block of one box's product at
 * one tree depth (kind 0 upward, 1 root, 2 downward); per tile: kind, depth,
 * first row, column count, and the times in microseconds from the earliest
 * claim at which it was claimed by a CTA or warp, its dependencies were met
 * and it was finished.  Arrays hold cap entries (any may be NULL); *count
 * receives the tile count.  RS_ERR_STATE if no such launch was profiled. */
int rs_profile_tiles(rs_handle h, int mode, int nrhs, int64_t cap, int* kind, int* depth, int* row0, int* ncol,
                     double* t_claim_us, double* t_start_us, double* t_end_us, int64_t* count);

/* FMA throughput of the current device, measured (not the paper's: a
 * roofline denominator for the FP64 and FP32 kernels): every thread runs 8
 * independent multiply-add chains, 8 CTAs of 256 threads per SM; the best of
 * three timed launches (CUDA events) after one warm-up.  precision
 * RS_PREC_FP64 or RS_PREC_FP32; *gflops receives 2 x FMAs / s / 1e9.  Allocates
 * and frees a small output buffer; synchronous. */
int rs_probe_fma_peak(int precision, double* gflops);

/* Self-test of the tensor-core building blocks the multi-column solve uses
 * (the paper has no counterpart): one block product D = A B^T on the
 * tensor cores (tcgen05.mma, cta_group::1, M = 128, operands staged in
 * shared memory in the 128-byte-swizzled K-major layout, accumulator in
 * tensor memory).  kind 0: A, B rounded to tf32, K = 32; kind 1: rounded to
 * bf16, K = 64.  A: 128 x K, B: n x K, D: 128 x n, all row-major fp32 in
 * DEVICE memory (caller-owned); n in {16, 32, ..., 256}.  Synchronous.
 * RS_ERR_ARG for bad arguments, RS_ERR_TIMEOUT if the MMA completion wait
 * ran out, RS_ERR_CUDA on a launch error. */
int rs_tc_selftest(int kind, const float* A, const float* B, float* D, int n);

/* Number of kernels the library has launched in this process so far
 * (measurement; no counterpart in the paper). */
int64_t rs_launch_count(void);

/* ------------------------------------------------------------------ serving
 * A server keeps factorizations resident and answers solve requests by
 * continuous batching (the paper has no serving layer; it motivates one:
 * Sec. 1 point (ii), many right-hand sides per factorization).  Every
 * registered handle gets a worker thread and a stream; the worker repeatedly
 * takes all requests queued for its handle (up to max_cols columns), packs
 * them into one batch, runs rs_solve_refined on it and completes each
 * request.  Requests arriving while a batch is on the GPU join the next
 * batch; different handles' columns are copied in and out concurrently, but
 * their solves take turns (one refined solve on the GPU at a time, each
 * filling the GPU).  Builds submitted
 * to the server run on a builder thread and are admitted only while the
 * estimated device memory of the resident factorizations plus the new one
 * stays under hbm_budget_bytes (<= 0: 90% of the free memory at creation);
 * an inadmissible build completes with RS_ERR_OOM.
 * B and X of a request are host buffers the caller keeps alive until the
 * request is waited for.  A handle registered with a server must not be
 * used directly while the server runs.  Latency = host time from submit to
 * completion. */
typedef struct rs_server_s* rs_server;
typedef struct {
  int64_t requests;        /* completed solve requests */
  int64_t rhs;             /* columns solved */
  int64_t batches;
  double mean_batch_cols;
  double p50_ms, p99_ms;   /* request latency percentiles */
  double elapsed_s;        /* since creation or the last reset */
  int handles;
  int64_t resident_bytes;  /* estimated device memory of the resident handles */
} rs_server_stats_t;

int rs_server_create(int max_cols, int64_t hbm_budget_bytes, rs_server* out);
/* Register a built handle (still owned by the caller); *handle_id names it. */
int rs_server_add_handle(rs_server s, rs_handle h, int* handle_id);
/* Queue a solve of ncols columns (tol: relative residual target). */
int rs_server_submit_solve(rs_server s, int handle_id, const void* B, int64_t ldb, int ncols,
                           void* X, int64_t ldx, double tol, int64_t* ticket);
/* Queue a build; on success the request's result is the new handle id.
 * pts (and, for RS_LAPLACE2D_DL, params->normals and params->curvature) are
 * host arrays copied at submission. */
int rs_server_submit_build(rs_server s, const double* pts, int64_t n, int dim,
                           const rs_params* params, double eps, int leaf, int64_t* ticket);
/* Wait (up to timeout_s; <= 0 waits indefinitely) for a request; status is
 * its rs_status, result the refinement count (solve) or the handle id
 * (build).  Each ticket can be waited for once. */
int rs_server_wait(rs_server s, int64_t ticket, double timeout_s, int* status,
                   double* latency_ms, double* relres, int* result);
int rs_server_stats(rs_server s, rs_server_stats_t* out);
int rs_server_reset_stats(rs_server s);
/* Handle behind an id (for builds made by the server). */
int rs_server_handle(rs_server s, int handle_id, rs_handle* out);
/* Drain the queues, stop the threads, free handles the server built. */
int rs_server_destroy(rs_server s);

/* Host-side fault injection for failure-path tests (no GPU fault is ever
 * caused):
 *   "alloc:n"  the n-th device allocation from now fails (RS_ERR_OOM);
 *   "wait"     the next solve's dependency waits target a round of tiles
 *              that never finishes, so the bounded spins run out, the kernel
 *              raises its flag and leaves, and the call returns
 *              RS_ERR_TIMEOUT; the next solve restarts its counters;
 *   "off" / NULL  disarm. */
int rs_set_fault(const char* spec);

/* Recursive skeletonization as a preconditioner (Sec. 6.4): solve a system
 * coupling npatch patches (scatterers) -- patch i's points X_i, its own
 * matrix A_ii = I + w_i K(X_i, X_i) and the couplings A_ij = w_j K(X_i, X_j)
 * (i != j), K_ii = 0 as everywhere -- by restarted GMRES(restart) with the
 * block-diagonal preconditioner diag(A_ii^-1), each block applied by patch
 * i's compressed inverse (FP64 solve).  The coupled matrix is applied densely
 * from the coordinates on the device (the paper uses an FMM there; that is
 * not part of this library), so n = sum of the patches' N should stay in the
 * tens of thousands.
 *   patches   npatch built handles (one per patch, same kernel, wavenumber
 *             and dimension; each built on exactly its patch's points, with
 *             its w); not modified
 *   pts       dim x n, point-major (point q at pts[q*dim ..]), the patches'
 *             points in patch order, each patch in the order it was built
 *             with; host or device
 *   B, X      n values (double, or interleaved complex for the Helmholtz
 *             kernels) in the same order; host or device; X is written
 *   tol       relative residual ||b - A x|| / ||b|| to reach (the true
 *             residual of the coupled matrix, checked at the end)
 *   max_it    total GMRES iterations allowed; restart: Krylov dimension
 *             (1..200); precondition: 0 runs plain GMRES (for comparison)
 *   its_out, relres_out (host, may be NULL): iterations used, final relative
 *             residual.  Returns RS_OK even when tol was not met.
 * Errors: RS_ERR_ARG (null or inconsistent arguments, the double layer), RS_ERR_OOM,
 * RS_ERR_CUDA, RS_ERR_TIMEOUT (a block solve's bounded wait ran out). */
int rs_gmres_patches(int npatch, const rs_handle* patches, const double* pts, const void* B, void* X,
                     double tol, int max_it, int restart, int precondition, int* its_out,
                     double* relres_out, void* stream);

/* Build-path override and path counters, for tests (the paper has no
 * counterpart: these select among this library's own kernels, all of which
 * compute the same ID and block elimination).  The multi-CTA forms of the ID
 * and of the Gauss-Jordan steps normally run only on boxes too large for
 * one CTA's shared memory (the top levels of the 3D workloads); the
 * override sends small problems through them too, so that they can be
 * compared with the oracle at sizes it finishes quickly.
 * rs_set_path(spec): comma-separated tokens, cumulative; NULL, "" or "off"
 * restores the normal selection:
 *   "id:big"      every ID level on the multi-CTA form (cluster first)
 *   "id:coop"     ... skipping the thread-block-cluster form
 *   "id:step"     ... skipping the cooperative form too (a launch per pivot step)
 *   "factor:big"  every factorization level on the multi-CTA form
 *   "gj:blocked"  Gauss-Jordan steps without the cluster form
 *   "gj:coop"     ... and without the blocked form
 *   "gj:step"     ... and without the cooperative form
 *   "tile:TMxTN"  every persistent solve of 16 or more columns on that tile
 *                 shape (32x32, 32x64, 64x32, 64x64: CUDA-core tiles;
 *                 128x64, 128x128, 128x256: tensor-core tiles, float
 *                 arithmetic on real kernels only -- elsewhere 32x64 is
 *                 used); "tile:warp" the warp kernel; by default the
 *                 autotuner picks per (mode, column count)
 * A form whose launch does not fit the device falls through to the next, as
 * in the normal selection.  RS_ERR_ARG for an unknown token.
 * rs_path_counts(counts, cap, reset): level launches per form since the last
 * reset, in the order ID {one CTA, cluster, cooperative, per step},
 * factorization {one CTA, multi-CTA, generic}, Gauss-Jordan {cluster,
 * blocked, cooperative, per step}; fills min(cap, total) entries of counts
 * (host), clears them if reset != 0, and returns the total number of
 * counters (11).  Process-wide. */
int rs_set_path(const char* spec);
int rs_path_counts(int64_t* counts, int cap, int reset);

/* Release every resource of the handle (device memory, workspaces, solve
 * plans) after the work queued on it has finished.  NULL is accepted.  Resource
 * management with no counterpart in the paper.  Returns RS_OK. */
int rs_free(rs_handle h);

/* Message of the calling thread's last error ("" if none); the string is the
 * library's (do not free), valid until the thread's next library call.  Error
 * reporting with no counterpart in the paper. */
const char* rs_last_error(void);

/* Library version string (static storage), e.g. "rs-gb300 0.1 (sm_103a)".
 * No counterpart in the paper. */
const char* rs_version(void);

/* The Green's function exactly as the library evaluates it (eqs. 2d-laplace,
 * 3d-laplace, 2d-helmholtz, 3d-helmholtz; no quadrature weight), at n squared
 * distances s2 > 0 (host array): out[n] for the real kernels, interleaved
 * (re, im) out[2 n] for the Helmholtz kernels (host).  For verification of the device evaluation
 * (2D Laplace uses a table-driven logarithm, Tang 1990); synchronous. */
int rs_green(int kernel_id, double k_wave, const double* s2, int64_t n, double* out);

#ifdef __cplusplus
}
#endif

#endif /* RS_H_ */
