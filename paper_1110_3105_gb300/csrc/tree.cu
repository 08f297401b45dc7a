// Tree: uniform quadtree / octree with contiguous index blocks.
//
// Sec. 2.1 (index tree of contiguous ranges), Example 1 (each box split
// into 2^d equal children, points reordered so every box is contiguous) and
// the opening of Sec. 6 (uniform subdivision to O(1) blocks, empty boxes
// dropped).  Root box: centre = midpoint of the bounding box, half-width
// a = 0.5 * largest extent * (1 + 2^-20).  Integer cell of a point per
// axis q = min(2^D - 1, floor((x - (c - a)) / (2a) * 2^D)) with D = 30 (2D),
// 20 (3D), computed with explicitly rounded double operations so it is
// bit-identical to any IEEE evaluation of the same expression.  Depth L =
// smallest depth at which every box holds <= leaf points; points ordered by
// (Morton key of the depth-L box, original index); boxes of each depth in
// Morton order; colleagues = same-depth boxes within one cell on every axis.
#include <algorithm>
#include <vector>

#include "rs_internal.h"

namespace rs {

namespace {

constexpr int BB_NT = 256;

// Bounding box partials: per block min/max of each axis.
__global__ void k_bbox_partial(const double* pts, int64_t n, int dim, double* part) {
  __shared__ double smin[3][BB_NT], smax[3][BB_NT];
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * BB_NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * BB_NT) {
    for (int d = 0; d < dim; ++d) {
      double v = pts[i * dim + d];
      if (!isfinite(v)) bad = 1;
      lo[d] = fmin(lo[d], v);
      hi[d] = fmax(hi[d], v);
    }
  }
  for (int d = 0; d < 3; ++d) {
    smin[d][threadIdx.x] = lo[d];
    smax[d][threadIdx.x] = bad ? NAN : hi[d];
  }
  __syncthreads();
  for (int o = BB_NT / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      for (int d = 0; d < 3; ++d) {
        smin[d][threadIdx.x] = fmin(smin[d][threadIdx.x], smin[d][threadIdx.x + o]);
        double a = smax[d][threadIdx.x], b = smax[d][threadIdx.x + o];
        smax[d][threadIdx.x] = (isnan(a) || isnan(b)) ? NAN : fmax(a, b);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int d = 0; d < 3; ++d) {
      part[blockIdx.x * 6 + d] = smin[d][0];
      part[blockIdx.x * 6 + 3 + d] = smax[d][0];
    }
}

// Root box from the partials: out = {c0, c1, c2, a, nonfinite flag}.
// One CTA of BB_NT threads: strided partial reductions, then a tree.
__global__ void k_root_box(const double* part, int nblk, int dim, double* out) {
  __shared__ double smin[3][BB_NT], smax[3][BB_NT];
  __shared__ int sbad;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  int bad = 0;
  if (threadIdx.x == 0) sbad = 0;
  for (int b = threadIdx.x; b < nblk; b += BB_NT)
    for (int d = 0; d < 3; ++d) {
      lo[d] = fmin(lo[d], part[b * 6 + d]);
      const double h = part[b * 6 + 3 + d];
      if (isnan(h)) bad = 1;
      hi[d] = fmax(hi[d], h);
    }
  for (int d = 0; d < 3; ++d) {
    smin[d][threadIdx.x] = lo[d];
    smax[d][threadIdx.x] = hi[d];
  }
  __syncthreads();
  if (bad) sbad = 1;
  for (int o = BB_NT / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int d = 0; d < 3; ++d) {
        smin[d][threadIdx.x] = fmin(smin[d][threadIdx.x], smin[d][threadIdx.x + o]);
        smax[d][threadIdx.x] = fmax(smax[d][threadIdx.x], smax[d][threadIdx.x + o]);
      }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  for (int d = 0; d < 3; ++d) {
    lo[d] = smin[d][0];
    hi[d] = smax[d][0];
  }
  bad = sbad;
  double ext = 0.0;
  for (int d = 0; d < dim; ++d) {
    out[d] = __dmul_rn(__dadd_rn(lo[d], hi[d]), 0.5);
    ext = fmax(ext, __dsub_rn(hi[d], lo[d]));
  }
  double a = ext > 0.0 ? __dmul_rn(__dmul_rn(ext, 0.5), 1.0 + 0x1p-20) : 1.0;
  out[3] = a;
  out[4] = bad ? 1.0 : 0.0;
}

__device__ inline uint64_t spread2(uint64_t v) {  // 30 bits -> every other bit
  v &= 0x3fffffffull;
  v = (v | (v << 16)) & 0x0000ffff0000ffffull;
  v = (v | (v << 8)) & 0x00ff00ff00ff00ffull;
  v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0full;
  v = (v | (v << 2)) & 0x3333333333333333ull;
  v = (v | (v << 1)) & 0x5555555555555555ull;
  return v;
}
__device__ inline uint64_t spread3(uint64_t v) {  // 20 bits -> every third bit
  v &= 0xfffffull;
  v = (v | (v << 32)) & 0x001f00000000ffffull;
  v = (v | (v << 16)) & 0x001f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}
__device__ inline uint64_t morton_key(const uint32_t* c, int dim) {
  if (dim == 2) return spread2(c[0]) | (spread2(c[1]) << 1);
  return spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2);
}
__device__ inline uint32_t compact2(uint64_t v) {
  v &= 0x5555555555555555ull;
  v = (v | (v >> 1)) & 0x3333333333333333ull;
  v = (v | (v >> 2)) & 0x0f0f0f0f0f0f0f0full;
  v = (v | (v >> 4)) & 0x00ff00ff00ff00ffull;
  v = (v | (v >> 8)) & 0x0000ffff0000ffffull;
  v = (v | (v >> 16)) & 0x00000000ffffffffull;
  return (uint32_t)v;
}
__device__ inline uint32_t compact3(uint64_t v) {
  v &= 0x1249249249249249ull;
  v = (v | (v >> 2)) & 0x10c30c30c30c30c3ull;
  v = (v | (v >> 4)) & 0x100f00f00f00f00full;
  v = (v | (v >> 8)) & 0x001f0000ff0000ffull;
  v = (v | (v >> 16)) & 0x001f00000000ffffull;
  v = (v | (v >> 32)) & 0x00000000000fffffull;
  return (uint32_t)v;
}

// Finest-cell Morton key of every point; vals = original index.
__global__ void k_keys(const double* pts, int64_t n, int dim, const double* box, int nbits, uint64_t* keys,
                       int* vals) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = box[3];
  double width = __dmul_rn(a, 2.0);
  double scale = (double)(1ull << nbits);
  uint32_t q[3] = {0, 0, 0};
  for (int d = 0; d < dim; ++d) {
    double lower = __dsub_rn(box[d], a);
    double t = __dmul_rn(__ddiv_rn(__dsub_rn(pts[i * dim + d], lower), width), scale);
    double f = floor(t);
    uint64_t qi = f < 0.0 ? 0ull : (uint64_t)f;
    uint64_t qmax = (1ull << nbits) - 1ull;
    q[d] = (uint32_t)(qi > qmax ? qmax : qi);
  }
  keys[i] = morton_key(q, dim);
  vals[i] = (int)i;
}

// For every depth l = 0..nbits: the largest number of points in one box.
// keys are sorted; a run start at depth l is where the depth-l prefix changes.
__global__ void k_level_occupancy(const uint64_t* keys, int n, int dim, int nbits, int* maxocc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int l = 0; l <= nbits; ++l) {
    int sh = dim * (nbits - l);
    uint64_t pre = sh >= 64 ? 0ull : (keys[i] >> sh);
    bool start = (i == 0) || ((sh >= 64 ? 0ull : (keys[i - 1] >> sh)) != pre);
    if (!start) continue;
    int lo = i, hi = n;  // first index with a different prefix
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      uint64_t pm = sh >= 64 ? 0ull : (keys[mid] >> sh);
      if (pm == pre) lo = mid; else hi = mid;
    }
    atomicMax(&maxocc[l], hi - i);
  }
}

__global__ void k_shift_keys(uint64_t* keys, int n, int sh) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) keys[i] = sh >= 64 ? 0ull : (keys[i] >> sh);
}

// Box-start flags at depth l from depth-L keys.
__global__ void k_box_flags(const uint64_t* keyL, int n, int sh, int* flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  flags[i] = (i == 0) || ((keyL[i] >> sh) != (keyL[i - 1] >> sh));
}

// Scatter box begins and per-point box index (pbox) from the scanned flags.
__global__ void k_box_begin(const int* flags, const int64_t* excl, int n, int* begin, int* pbox) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int b = (int)excl[i] + flags[i] - 1;
  pbox[i] = b;
  if (flags[i]) begin[b] = i;
}

__global__ void k_box_info(const uint64_t* keyL, const int* begin, int nbox, int dim, int sh, uint64_t* keys,
                           int* coords, const int* pbox_up, int* parent) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  uint64_t k = keyL[begin[b]] >> sh;
  keys[b] = k;
  if (dim == 2) {
    coords[b * 2 + 0] = (int)compact2(k);
    coords[b * 2 + 1] = (int)compact2(k >> 1);
  } else {
    coords[b * 3 + 0] = (int)compact3(k);
    coords[b * 3 + 1] = (int)compact3(k >> 1);
    coords[b * 3 + 2] = (int)compact3(k >> 2);
  }
  parent[b] = pbox_up ? pbox_up[begin[b]] : -1;
}

__global__ void k_child_ranges(const int* parent_of_child, int nchild, int* child_begin, int* child_end) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchild) return;
  int p = parent_of_child[c];
  if (c == 0 || parent_of_child[c - 1] != p) child_begin[p] = c;
  if (c == nchild - 1 || parent_of_child[c + 1] != p) child_end[p] = c + 1;
}

__global__ void k_colleagues(const uint64_t* keys, const int* coords, int nbox, int dim, int depth, int* ncoll,
                             int* coll) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  int lim = 1 << depth;
  int found[26];
  int nf = 0;
  int noff = dim == 2 ? 9 : 27;
  for (int o = 0; o < noff; ++o) {
    int off[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
    if (dim == 2) off[2] = 0;
    if (off[0] == 0 && off[1] == 0 && off[2] == 0) continue;
    uint32_t c[3];
    bool ok = true;
    for (int d = 0; d < dim; ++d) {
      int v = coords[b * dim + d] + off[d];
      if (v < 0 || v >= lim) ok = false;
      c[d] = (uint32_t)v;
    }
    if (!ok) continue;
    uint64_t key = morton_key(c, dim);
    int lo = 0, hi = nbox;  // lower bound
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    if (lo < nbox && keys[lo] == key) found[nf++] = lo;
  }
  for (int i = 1; i < nf; ++i) {  // insertion sort, ascending box index
    int v = found[i], j = i - 1;
    while (j >= 0 && found[j] > v) { found[j + 1] = found[j]; --j; }
    found[j + 1] = v;
  }
  ncoll[b] = nf;
  for (int i = 0; i < 27; ++i) coll[b * 27 + i] = i < nf ? found[i] : -1;
}

// Points in tree order, one block per axis.
__global__ void k_permute_points(const double* pts, const int* perm, int64_t n, int dim, double* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t src = perm[i];
  for (int d = 0; d < dim; ++d) out[d * n + i] = pts[src * dim + d];
}

// Box count of one depth: last exclusive prefix + last flag.
__global__ void k_count(const int* flags, const int64_t* excl, int n, int64_t* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = excl[n - 1] + flags[n - 1];
}

// Pinned host staging for the device -> host copies of a build (one per
// host thread, grown as needed and kept).
struct PinnedStage {
  void* p = nullptr;
  size_t cap = 0;
};
static thread_local PinnedStage tl_stage;
static int stage_reserve(size_t bytes, void** out) {
  if (bytes > tl_stage.cap) {
    if (tl_stage.p) cudaFreeHost(tl_stage.p);
    tl_stage.p = nullptr;
    tl_stage.cap = 0;
    const size_t want = std::max<size_t>(bytes, 4u << 20);
    RS_CUDA(cudaMallocHost(&tl_stage.p, want));
    tl_stage.cap = want;
  }
  *out = tl_stage.p;
  return RS_OK;
}

__global__ void k_iota(int* a, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = i;
}

}  // namespace

int build_tree(Handle* h, const double* d_pts_in, cudaStream_t st) {
  const int n = (int)h->N, dim = h->dim;
  const int nbits = dim == 2 ? 30 : 20;
  const int NT = 256;
  const int nb = div_up(n, NT);

  prof_begin(P_TREE, st);
  // root box
  int nblk = std::min(nb, 1024);
  double* part = nullptr;
  double* box = nullptr;
  RS_TRY(dalloc_t(h, &part, (size_t)nblk * 6));
  RS_TRY(dalloc_t(h, &box, 8));
  k_bbox_partial<<<nblk, BB_NT, 0, st>>>(d_pts_in, n, dim, part);
  RS_CHECK_LAUNCH();
  k_root_box<<<1, BB_NT, 0, st>>>(part, nblk, dim, box);
  RS_CHECK_LAUNCH();
  double hbox[5];
  RS_CUDA(cudaMemcpyAsync(hbox, box, sizeof(hbox), cudaMemcpyDeviceToHost, st));
  RS_CUDA(cudaStreamSynchronize(st));
  if (hbox[4] != 0.0) return fail(RS_ERR_NAN, "rs_build: non-finite point coordinate");
  for (int d = 0; d < 3; ++d) h->center[d] = d < dim ? hbox[d] : 0.0;
  h->half = hbox[3];

  // keys, sort by the finest key, depth from occupancy
  uint64_t *keys, *keys2;
  int *vals, *vals2;
  RS_TRY(dalloc_t(h, &keys, n));
  RS_TRY(dalloc_t(h, &keys2, n));
  RS_TRY(dalloc_t(h, &vals, n));
  RS_TRY(dalloc_t(h, &vals2, n));
  k_keys<<<nb, NT, 0, st>>>(d_pts_in, n, dim, box, nbits, keys, vals);
  RS_CHECK_LAUNCH();
  uint64_t* skeys;
  int* svals;
  RS_TRY(dalloc_t(h, &skeys, n));
  RS_TRY(dalloc_t(h, &svals, n));
  // Depth from the occupancy of every depth's boxes: sort by the top key bits
  // first (the depths whose prefixes they hold), all bits only if no depth
  // up to there is fine enough.
  int* maxocc;
  RS_TRY(dalloc_t(h, &maxocc, nbits + 1));
  std::vector<int> occ(nbits + 1);
  int L = -1;
  const int top_levels = std::min(nbits, 32 / dim);
  for (int pass = 0; pass < 2 && L < 0; ++pass) {
    const int lv_top = pass == 0 ? top_levels : nbits;
    if (pass == 1 && top_levels == nbits) break;
    RS_CUDA(cudaMemcpyAsync(skeys, keys, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st));
    RS_CUDA(cudaMemcpyAsync(svals, vals, sizeof(int) * n, cudaMemcpyDeviceToDevice, st));
    if (lv_top < nbits) {
      k_shift_keys<<<nb, NT, 0, st>>>(skeys, n, dim * (nbits - lv_top));
      RS_CHECK_LAUNCH();
    }
    RS_TRY(radix_sort_pairs(skeys, svals, keys2, vals2, n, dim * lv_top, st));
    RS_CUDA(cudaMemsetAsync(maxocc, 0, sizeof(int) * (nbits + 1), st));
    k_level_occupancy<<<nb, NT, 0, st>>>(skeys, n, dim, lv_top, maxocc);
    RS_CHECK_LAUNCH();
    RS_CUDA(cudaMemcpyAsync(occ.data(), maxocc, sizeof(int) * (lv_top + 1), cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaStreamSynchronize(st));
    for (int l = 0; l <= lv_top; ++l)
      if (occ[l] <= h->leaf) { L = l; break; }
  }
  if (L < 0) return fail(RS_ERR_ARG, "rs_build: more than leaf=%d coincident points", h->leaf);
  h->L = L;

  // stable sort of (depth-L key, original index) from the original order
  k_shift_keys<<<nb, NT, 0, st>>>(keys, n, dim * (nbits - L));
  RS_CHECK_LAUNCH();
  RS_TRY(radix_sort_pairs(keys, vals, keys2, vals2, n, dim * L, st));
  h->perm = vals;
  RS_TRY(dalloc_t(h, &h->pts, (size_t)3 * n));
  RS_CUDA(cudaMemsetAsync(h->pts, 0, sizeof(double) * 3 * (size_t)n, st));
  k_permute_points<<<nb, NT, 0, st>>>(d_pts_in, vals, n, dim, h->pts);
  RS_CHECK_LAUNCH();

  // box tables for every depth: start flags and their scans for all depths,
  // then one host read of the box counts
  h->lv.assign(L + 1, Level());
  int *flags, *pbox_prev = nullptr;
  int64_t *excl, *counts;
  RS_TRY(dalloc_t(h, &flags, (size_t)n * (L + 1)));
  RS_TRY(dalloc_t(h, &excl, (size_t)n * (L + 1)));
  RS_TRY(dalloc_t(h, &counts, L + 1));
  for (int l = 0; l <= L; ++l) {
    k_box_flags<<<nb, NT, 0, st>>>(keys, n, dim * (L - l), flags + (size_t)l * n);
    RS_CHECK_LAUNCH();
    RS_TRY(scan_i32_to_i64(flags + (size_t)l * n, excl + (size_t)l * n, n, nullptr, st));
    k_count<<<1, 32, 0, st>>>(flags + (size_t)l * n, excl + (size_t)l * n, n, counts + l);
    RS_CHECK_LAUNCH();
  }
  std::vector<int64_t> nboxes(L + 1);
  RS_CUDA(cudaMemcpyAsync(nboxes.data(), counts, sizeof(int64_t) * (L + 1), cudaMemcpyDeviceToHost, st));
  RS_CUDA(cudaStreamSynchronize(st));
  size_t host_ints = 0;
  for (int l = 0; l <= L; ++l) host_ints += (size_t)nboxes[l] * 30;
  void* pin = nullptr;
  RS_TRY(stage_reserve(sizeof(int) * std::max<size_t>(1, host_ints), &pin));
  int* hp = (int*)pin;
  for (int l = 0; l <= L; ++l) {
    Level& lv = h->lv[l];
    lv.depth = l;
    int sh = dim * (L - l);
    const int64_t nbox = nboxes[l];
    const int* fl = flags + (size_t)l * n;
    const int64_t* ex = excl + (size_t)l * n;
    lv.nbox = (int)nbox;
    int* pbox;
    RS_TRY(dalloc_t(h, &pbox, n));
    RS_TRY(dalloc_t(h, &lv.begin, nbox));
    RS_TRY(dalloc_t(h, &lv.parent, nbox));
    RS_TRY(dalloc_t(h, &lv.child_begin, nbox));
    RS_TRY(dalloc_t(h, &lv.child_end, nbox));
    RS_TRY(dalloc_t(h, &lv.ncoll, nbox));
    RS_TRY(dalloc_t(h, &lv.coll, nbox * 27));
    RS_TRY(dalloc_t(h, &lv.coords, nbox * dim));
    RS_TRY(dalloc_t(h, &lv.keys, nbox));
    k_box_begin<<<nb, NT, 0, st>>>(fl, ex, n, lv.begin, pbox);
    RS_CHECK_LAUNCH();
    int bb = div_up(nbox, NT);
    k_box_info<<<bb, NT, 0, st>>>(keys, lv.begin, (int)nbox, dim, sh, lv.keys, lv.coords, pbox_prev, lv.parent);
    RS_CHECK_LAUNCH();
    RS_CUDA(cudaMemsetAsync(lv.child_begin, 0, sizeof(int) * nbox, st));
    RS_CUDA(cudaMemsetAsync(lv.child_end, 0, sizeof(int) * nbox, st));
    if (l > 0) {
      k_child_ranges<<<bb, NT, 0, st>>>(lv.parent, (int)nbox, h->lv[l - 1].child_begin, h->lv[l - 1].child_end);
      RS_CHECK_LAUNCH();
    }
    k_colleagues<<<bb, NT, 0, st>>>(lv.keys, lv.coords, (int)nbox, dim, l, lv.ncoll, lv.coll);
    RS_CHECK_LAUNCH();
    pbox_prev = pbox;
    // host copies for sizing and inspection, staged in pinned memory
    RS_CUDA(cudaMemcpyAsync(hp, lv.begin, sizeof(int) * nbox, cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaMemcpyAsync(hp + nbox, lv.parent, sizeof(int) * nbox, cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaMemcpyAsync(hp + 2 * nbox, lv.ncoll, sizeof(int) * nbox, cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaMemcpyAsync(hp + 3 * nbox, lv.coll, sizeof(int) * nbox * 27, cudaMemcpyDeviceToHost, st));
    hp += 30 * nbox;
  }
  RS_CUDA(cudaStreamSynchronize(st));
  hp = (int*)pin;
  for (int l = 0; l <= L; ++l) {
    Level& lv = h->lv[l];
    const int64_t nbox = lv.nbox;
    lv.h_begin.assign(hp, hp + nbox);
    lv.h_parent.assign(hp + nbox, hp + 2 * nbox);
    lv.h_ncoll.assign(hp + 2 * nbox, hp + 3 * nbox);
    lv.h_coll.assign(hp + 3 * nbox, hp + 30 * nbox);
    hp += 30 * nbox;
  }

  // leaf active sets: identity
  Level& leaf = h->lv[L];
  RS_TRY(dalloc_t(h, &leaf.act, n));
  k_iota<<<nb, NT, 0, st>>>(leaf.act, n);
  RS_CHECK_LAUNCH();
  prof_end(P_TREE, st, (double)n * dim * 8.0, 0.0);
  return RS_OK;
}

}  // namespace rs
