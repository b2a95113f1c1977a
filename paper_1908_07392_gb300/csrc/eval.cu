// Evaluation engine: vp_tree_upload, vp_eval, vp_eval_host and friends.
//
// Every step of the volume potential is a set of small dense contractions
// y_dst (=|+=) A_op x_src, where A_op is a precomputed operator chosen by
// (level, relative position) and x_src / y_dst are per-box vectors (nodal
// values, multipole or local coefficients). The planner groups the
// contractions by operator so that each group is one GEMM whose columns are
// gathered from (and scattered to) arbitrary vectors; several destinations
// that receive more than one contribution get private scratch slots that a
// deterministic segmented reduction sums in a fixed order afterwards.
//
// Pass order (one stream):
//   S2M (leaves) -> M2M (deepest parent level first) -> M2L (V lists) and
//   S2L (X lists) into local slots -> reduce into local expansions ->
//   L2L (coarsest first) -> L2T, M2T (W lists) and near tables (U lists) into
//   output slots -> reduce into u, du/dx, du/dy.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <new>
#include <vector>

#include "layer.h"
#include "plan.h"
#include "special.cuh"
#include "split.h"
#include "vp_internal.h"

namespace vp {

enum Buf { BUF_F = 0, BUF_MP, BUF_LOC, BUF_LSLOT, BUF_USLOT, BUF_COUNT };

struct Tile {
  int group, m0, col0, ncol;
};

struct GemmArgs {
  int M, K, kseg, lda, accumulate;
  long long seg_stride;
  const double* A;
  const double* X;
  double* Y;
  const Tile* tiles;
  const long long* a_off;
  const long long* src_off;
  const long long* dst_off;
};

// FP64 gather-GEMM: tile (64 rows x 64 columns), K in steps of 16, 256 threads,
// each thread 4 rows (strided by 16) x 4 columns; rows of a destination vector
// are contiguous, so a half-warp stores 16 consecutive doubles.
constexpr int kBM = 64, kBN = 64, kBK = 16;

// Deepest leaf level vp_tree_interp serves (its cell map holds 4^L ints: 256 MB at L = 13).
constexpr int kInterpMaxLevel = 13;

// TAG only names the instantiation (1: near-field tables) so profilers can pick it out.
template <int TAG>
__global__ void __launch_bounds__(256) k_gemm_gather_f64(GemmArgs a) {
  __shared__ double As[kBK][kBM + 2];
  __shared__ double Bs[kBK][kBN + 2];
  const Tile tile = a.tiles[blockIdx.x];
  const double* __restrict__ A = a.A + a.a_off[tile.group];
  const int tid = threadIdx.x;
  const int tr = tid & 15;   // row lane
  const int tc = tid >> 4;   // column group (0..15)
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int k0 = 0; k0 < a.K; k0 += kBK) {
    // A tile: 64 rows x 16 k
    for (int e = tid; e < kBM * kBK; e += 256) {
      const int r = e / kBK, kk = e % kBK;
      const int gm = tile.m0 + r, gk = k0 + kk;
      As[kk][r] = (gm < a.M && gk < a.K) ? A[(size_t)gm * a.lda + gk] : 0.0;
    }
    // B tile: 16 k x 64 columns, gathered
    for (int e = tid; e < kBN * kBK; e += 256) {
      const int c = e / kBK, kk = e % kBK;
      const int gk = k0 + kk;
      double v = 0.0;
      if (c < tile.ncol && gk < a.K) {
        const long long base = a.src_off[tile.col0 + c];
        const int sg = gk / a.kseg, si = gk - sg * a.kseg;
        v = a.X[base + sg * a.seg_stride + si];
      }
      Bs[kk][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][tr + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tc * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = tc * 4 + j;
    if (c >= tile.ncol) continue;
    double* __restrict__ y = a.Y + a.dst_off[tile.col0 + c];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = tile.m0 + tr + 16 * i;
      if (r < a.M) y[r] = a.accumulate ? y[r] + acc[i][j] : acc[i][j];
    }
  }
}

struct ReduceArgs {
  int M, n;               // vector length; nodes per leaf (final output)
  int final_out;          // 1: write u / gradu layout
  long long N;            // nodes (final output)
  const long long* dst_off;
  const long long* ptr;   // CSR over destinations
  const long long* slot;  // scratch offsets
  const double* S;        // scratch base
  double* Y;              // destination base (non-final)
  double* u;              // final: u [N]
  double* g;              // final: gradu [2][N]
};

__global__ void k_reduce(ReduceArgs a) {
  constexpr int kChunk = 64;  // slot offsets staged in shared memory per pass
  __shared__ long long slot_sh[kChunk];
  const int d = blockIdx.x;
  const long long b = a.ptr[d], e = a.ptr[d + 1];
  const int rows_per_pass = (a.M + blockDim.x - 1) / blockDim.x;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};  // rows threadIdx.x + q blockDim.x, summed in slot order
  for (long long c0 = b; c0 < e; c0 += kChunk) {
    const int nc = (int)((e - c0) < kChunk ? (e - c0) : kChunk);
    __syncthreads();
    if (threadIdx.x < nc) slot_sh[threadIdx.x] = a.slot[c0 + threadIdx.x];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q >= rows_per_pass) break;
      const int r = threadIdx.x + q * blockDim.x;
      if (r >= a.M) break;
      int k = 0;
      for (; k + 4 <= nc; k += 4) {
        const double v0 = a.S[slot_sh[k] + r], v1 = a.S[slot_sh[k + 1] + r];
        const double v2 = a.S[slot_sh[k + 2] + r], v3 = a.S[slot_sh[k + 3] + r];
        acc[q] += v0; acc[q] += v1; acc[q] += v2; acc[q] += v3;
      }
      for (; k < nc; ++k) acc[q] += a.S[slot_sh[k] + r];
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = threadIdx.x + q * blockDim.x;
    if (q >= rows_per_pass || r >= a.M) break;
    const double s = acc[q];
    if (a.final_out) {
      const int f = r / a.n, t = r - f * a.n;
      const long long o = a.dst_off[d] + t;  // leaf * n + t
      if (f == 0) a.u[o] = s;
      else a.g[(f - 1) * a.N + o] = s;
    } else {
      a.Y[a.dst_off[d] + r] = s;
    }
  }
}

__global__ void k_nodes(int p, int n_leaves, double x0, double y0, double side, const int* lv, const int* ix,
                        const int* iy, const double* xi, long long N, double* xy) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int n = p * p;
  const long long leaf = i / n;
  const int t = (int)(i - leaf * n);
  const double h = side / (double)(1ll << lv[leaf]);
  xy[i] = x0 + (ix[leaf] + 0.5 * (1.0 + xi[t % p])) * h;
  xy[N + i] = y0 + (iy[leaf] + 0.5 * (1.0 + xi[t / p])) * h;
}

// Cell map at the finest level L: the leaves tile the root box, so each of the 4^L cells is
// covered by exactly one leaf, written by that leaf's block.
__global__ void k_cell_map(int n_leaves, int L, const int* lv, const int* ix, const int* iy, int* cell) {
  const int leaf = blockIdx.x;
  if (leaf >= n_leaves) return;
  const int sh = L - lv[leaf];
  const long long w = 1ll << sh, dim = 1ll << L;
  const long long x0 = (long long)ix[leaf] << sh, y0 = (long long)iy[leaf] << sh;
  for (long long k = threadIdx.x; k < w * w; k += blockDim.x) cell[(y0 + k / w) * dim + x0 + k % w] = leaf;
}

// Lagrange basis on the p Gauss-Legendre nodes at t (product form; exact 0/1 at the nodes).
__device__ inline void lagrange_basis(int p, const double* xi, double t, double* l) {
  for (int i = 0; i < p; ++i) {
    double v = 1.0;
    for (int k = 0; k < p; ++k)
      if (k != i) v *= (t - xi[k]) / (xi[i] - xi[k]);
    l[i] = v;
  }
}

// One thread per point: locate the leaf, evaluate the leaf's tensor interpolant of each field.
__global__ void k_interp(int p, int L, double x0, double y0, double side, const int* lv, const int* ix,
                        const int* iy, const double* xi_g, const int* cell, int n_fields, const double* F,
                        long long N, int M, const double* pts, double* out) {
  __shared__ double xi[16];
  if (threadIdx.x < p) xi[threadIdx.x] = xi_g[threadIdx.x];
  __syncthreads();
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const double px = pts[m], py = pts[(long long)M + m];
  const long long dim = 1ll << L;
  const double sx = (px - x0) / side * (double)dim, sy = (py - y0) / side * (double)dim;
  if (!(sx >= 0.0 && sx <= (double)dim && sy >= 0.0 && sy <= (double)dim)) {
    for (int f = 0; f < n_fields; ++f) out[(long long)f * M + m] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  const long long cx = min((long long)sx, dim - 1), cy = min((long long)sy, dim - 1);
  const int leaf = cell[cy * dim + cx];
  const double h = side / (double)(1ll << lv[leaf]);
  const double tx = 2.0 * ((px - x0) / h - ix[leaf]) - 1.0, ty = 2.0 * ((py - y0) / h - iy[leaf]) - 1.0;
  double lx[16], ly[16];
  lagrange_basis(p, xi, tx, lx);
  lagrange_basis(p, xi, ty, ly);
  const long long base = (long long)leaf * p * p;
  for (int f = 0; f < n_fields; ++f) {
    const double* v = F + (long long)f * N + base;
    double acc = 0.0;
    for (int j = 0; j < p; ++j) {
      double row = 0.0;
      for (int i = 0; i < p; ++i) row = fma(lx[i], v[j * p + i], row);
      acc = fma(ly[j], row, acc);
    }
    out[(long long)f * M + m] = acc;
  }
}

// ----------------------------------------------------------------- host plan -> device ops

struct HostGemm {
  int M = 0, K = 0, kseg = 0, lda = 0, accumulate = 0;
  long long seg_stride = 0;
  int table = 0;  // which table array
  int src = 0, dst = 0;
  // split precision: source vector family (-1: always FP64; 0: leaf values, 1: (box, channel)
  // multipoles, 2: box locals) and output (0: double-float slot, 1: FP64 overwrite, 2: FP64 accumulate)
  int split_vec = -1, out_mode = 0;
  long long mat_elems = 0;  // elements of one operator matrix (0: M * lda; set when M is a leading part)
  struct Entry { long long a, s, d, v = -1; };  // v: sliced-vector id (split), -1 = derived from s
  std::vector<Entry> entries;
};

struct DevGemm {
  GemmArgs args;
  int src, dst, table;
  int n_tiles;
};

struct HostReduce {
  int M = 0, final_out = 0, dst = 0, src = 0;
  std::vector<long long> dst_off, ptr, slot;
};

struct DevReduce {
  ReduceArgs args;
  int dst, src, n_dst;
};

struct DevSplit {
  SplitArgs args;
  int table, vec, dst;
  const SplitTile* tiles[kEngines];  // tile lists of the engines
  int n_tiles[kEngines];
  int engine = kEngineMmaSync;  // chosen per launch (vp_tree_set_engine, vp_autotune)
};

// Sliced-vector families (split precision): 0 leaf values (K = n), 1 (box, channel) multipoles (K = C),
// 2 box locals (K = E), 3 multipoles of children 0-1 of (parent, channel) (K = 2C), 4 (box, channel)
// locals (K = C), 5 multipoles of children 2-3 of (parent, channel) (K = 2C).
constexpr int kVecFamilies = 6;
struct DevSlice {
  int family, buf, K, kseg;
  long long seg_stride, cstride, n;
  const long long* base;  // null: contiguous, b = v * cstride
  const long long* vid;   // null: identity
};

enum Table { T_NEAR, T_S2M, T_L2T, T_M2M, T_L2L, T_M2L, T_M2T, T_S2L, T_M2M_LO, T_M2M_HI };

// A point-source operator launch (layer potential): instances of small dense matrices applied to the
// boundary density (layer.h), written into buffer `dst`.
struct DevPt {
  PtInst* inst = nullptr;
  int n_inst = 0, rows = 0, rb = 0, dst = 0;
  long long bs = 0;
  double* A = nullptr;
};

// Near-boundary corrections of a layer program: per corrected node its (node, panel) pairs (CSR) and
// the weight differences (layer.h).
struct DevNear {
  long long n_nodes = 0, n_pairs = 0;
  long long *node = nullptr, *ptr = nullptr;
  int* panel = nullptr;
  double* dW = nullptr;
};

struct Step {
  int kind;   // 0 gemm, 1 reduce, 2 memset mp, 3 slice vectors, 4 split gemm, 5 double-float reduce,
              // 6 point-source operator, 7 near-boundary correction of the output
  int index;
  int stage;  // VP_STAGE_* for timing
  double flops = 0.0;  // algorithmic floating-point operations of the step
  double bytes = 0.0;  // algorithmic device-memory bytes: every operand read once, every output written once
};

}  // namespace vp

struct vp_tree_s {
  vp_tables_s* T = nullptr;
  int n_leaves = 0, n_boxes = 0, max_level = 0;
  long long N = 0;
  double cx = 0.0, cy = 0.0;
  // device
  int *d_lv = nullptr, *d_ix = nullptr, *d_iy = nullptr;
  double* d_xi = nullptr;
  double *mp = nullptr, *loc = nullptr, *lslot = nullptr, *uslot = nullptr;
  long long n_lslot = 0, n_uslot = 0;
  int lslot_stride = 0, uslot_stride = 0;  // slot strides of a layer program (even: 16-byte aligned slots)
  std::vector<void*> allocs;  // every device allocation owned by the tree
  std::vector<vp::DevGemm> gemms;
  std::vector<vp::DevReduce> reduces;
  std::vector<vp::Step> steps;
  int cur_stage = 0;        // stage tag given to steps as they are planned
  double flops[VP_NSTAGES] = {0};
  double bytes[VP_NSTAGES] = {0};
  // split precision: sliced source vectors (leaf values, multipoles, locals) and their exponents
  std::vector<vp::DevSplit> splits;
  void* sv[vp::kVecFamilies] = {nullptr};
  int* se[vp::kVecFamilies] = {nullptr};
  std::vector<vp::DevSlice> slice_ops;
  // host staging for vp_eval_host
  double *h_f = nullptr, *h_u = nullptr;
  double *d_f = nullptr, *d_u = nullptr, *d_g = nullptr;
  // point location for vp_tree_interp: finest-level cell -> leaf, built on first use
  int* d_cell = nullptr;
  // host copy of the leaf list (level, ix, iy), kept for programs built later on the same tree
  std::vector<int> h_lv, h_ix, h_iy;
  // layer-potential program: multipole buffer size (0: n_boxes * E), point-source operators and
  // the source permutation they read the density through
  long long mp_elems = 0;
  std::vector<vp::DevPt> pts;
  std::vector<vp::DevNear> nears;
  int* d_perm = nullptr;
  // overlap of the near field with the far-field chain (vp_eval): the chain runs on `side`, a
  // high-priority stream, the near field on the caller's stream; events fork and join them
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_src = nullptr, ev_join = nullptr;
};

namespace vp {
namespace {

#define TRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_last_cuda(e_); return e_ == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA; } } while (0)

template <class T>
int dev_upload(vp_tree_s* tr, const std::vector<T>& v, T** out, cudaStream_t s) {
  *out = nullptr;
  if (v.empty()) return VP_OK;
  void* p = nullptr;
  TRY(cudaMalloc(&p, v.size() * sizeof(T)));
  tr->allocs.push_back(p);
  TRY(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  *out = static_cast<T*>(p);
  return VP_OK;
}

int upload_split(vp_tree_s* tr, HostGemm& g, cudaStream_t s);

// Number of distinct values in v.
long long count_distinct(std::vector<long long> v) {
  std::sort(v.begin(), v.end());
  return (long long)(std::unique(v.begin(), v.end()) - v.begin());
}

int upload_gemm(vp_tree_s* tr, HostGemm& g, cudaStream_t s) {
  if (g.entries.empty()) return VP_OK;
  if (tr->T->precision == VP_PREC_SPLIT && g.split_vec >= 0) return upload_split(tr, g, s);
  std::stable_sort(g.entries.begin(), g.entries.end(),
                   [](const HostGemm::Entry& x, const HostGemm::Entry& y) { return x.a < y.a; });
  std::vector<long long> a_off, src_off, dst_off;
  std::vector<Tile> tiles;
  size_t i = 0;
  while (i < g.entries.size()) {
    size_t j = i;
    while (j < g.entries.size() && g.entries[j].a == g.entries[i].a) ++j;
    const int grp = (int)a_off.size();
    a_off.push_back(g.entries[i].a);
    const int col_begin = (int)src_off.size();
    for (size_t k = i; k < j; ++k) { src_off.push_back(g.entries[k].s); dst_off.push_back(g.entries[k].d); }
    const int ncols = (int)(j - i);
    for (int m0 = 0; m0 < g.M; m0 += kBM)
      for (int c0 = 0; c0 < ncols; c0 += kBN) tiles.push_back({grp, m0, col_begin + c0, std::min(kBN, ncols - c0)});
    i = j;
  }
  DevGemm d{};
  d.args.M = g.M; d.args.K = g.K; d.args.kseg = g.kseg ? g.kseg : g.K; d.args.lda = g.lda;
  d.args.accumulate = g.accumulate; d.args.seg_stride = g.seg_stride;
  Tile* dt; long long *da, *ds, *dd;
  int rc;
  if ((rc = dev_upload(tr, tiles, &dt, s))) return rc;
  if ((rc = dev_upload(tr, a_off, &da, s))) return rc;
  if ((rc = dev_upload(tr, src_off, &ds, s))) return rc;
  if ((rc = dev_upload(tr, dst_off, &dd, s))) return rc;
  d.args.tiles = dt; d.args.a_off = da; d.args.src_off = ds; d.args.dst_off = dd;
  d.src = g.src; d.dst = g.dst; d.table = g.table; d.n_tiles = (int)tiles.size();
  // algorithmic bytes: each operator and each distinct source vector read once, each output column
  // written once (read as well when accumulating)
  const double fl = 2.0 * g.M * (double)g.K * (double)g.entries.size();
  const double by = 8.0 * ((double)a_off.size() * g.M * g.K + (double)count_distinct(src_off) * g.K +
                           (1.0 + g.accumulate) * (double)g.entries.size() * g.M);
  tr->steps.push_back({0, (int)tr->gemms.size(), tr->cur_stage, fl, by});
  tr->gemms.push_back(d);
  tr->flops[tr->cur_stage] += fl;
  tr->bytes[tr->cur_stage] += by;
  return VP_OK;
}

// Split-precision contraction: the same grouping, with tiles of the tensor-core kernel, matrix indices
// instead of element offsets and vector indices instead of source offsets.
int upload_split(vp_tree_s* tr, HostGemm& g, cudaStream_t s) {
  const vp_tables_s* T = tr->T;
  std::stable_sort(g.entries.begin(), g.entries.end(),
                   [](const HostGemm::Entry& x, const HostGemm::Entry& y) { return x.a < y.a; });
  const long long mat_elems = g.mat_elems ? g.mat_elems : (long long)g.M * g.lda;
  const long long vec_len = g.split_vec == 0 ? T->n : (g.split_vec == 1 ? T->C : T->E);  // families 0-2
  std::vector<long long> a_mat, src_vec, dst_off;
  std::vector<SplitTile> tiles[kEngines];
  size_t i = 0;
  while (i < g.entries.size()) {
    size_t j = i;
    while (j < g.entries.size() && g.entries[j].a == g.entries[i].a) ++j;
    const int grp = (int)a_mat.size();
    a_mat.push_back(g.entries[i].a / mat_elems);
    const int col_begin = (int)src_vec.size();
    for (size_t k = i; k < j; ++k) {
      src_vec.push_back(g.entries[k].v >= 0 ? g.entries[k].v : g.entries[k].s / vec_len);
      dst_off.push_back(g.entries[k].d);
    }
    const int ncols = (int)(j - i);
    // the row tiles of one column block are consecutive, so the CTAs that run them at the same time
    // share the block's gathered source columns in L2
    for (int en = 0; en < kEngines; ++en)
      for (int c0 = 0; c0 < ncols; c0 += kSplitBN[en])
        for (int m0 = 0; m0 < g.M; m0 += kSplitBMe[en])
          tiles[en].push_back({grp, m0, col_begin + c0, std::min(kSplitBN[en], ncols - c0)});
    i = j;
  }
  DevSplit d{};
  d.args.M = g.M; d.args.Kpad = split_kpad(g.K); d.args.out_mode = g.out_mode;
  long long *da, *ds, *dd;
  int rc;
  for (int en = 0; en < kEngines; ++en) {
    SplitTile* dt = nullptr;
    if ((rc = dev_upload(tr, tiles[en], &dt, s))) return rc;
    d.tiles[en] = dt;
    d.n_tiles[en] = (int)tiles[en].size();
  }
  if ((rc = dev_upload(tr, a_mat, &da, s))) return rc;
  if ((rc = dev_upload(tr, src_vec, &ds, s))) return rc;
  if ((rc = dev_upload(tr, dst_off, &dd, s))) return rc;
  d.args.a_mat = da; d.args.src_vec = ds; d.args.dst_off = dd;
  d.table = g.table; d.vec = g.split_vec; d.dst = g.dst;
  // algorithmic bytes: sliced operators (S bf16 slices + a row exponent) and sliced source vectors
  // (S slices + an exponent) read once, outputs written once (8 bytes: a double-float slot or FP64)
  const int kp = split_kpad(g.K);
  const double fl = 2.0 * g.M * (double)g.K * (double)g.entries.size();
  const double by = (double)a_mat.size() * g.M * (2.0 * kSplitSlices * kp + 4.0) +
                    (double)count_distinct(src_vec) * (2.0 * kSplitSlices * kp + 4.0) +
                    8.0 * (1.0 + (g.out_mode == 2)) * (double)g.entries.size() * g.M;
  tr->steps.push_back({4, (int)tr->splits.size(), tr->cur_stage, fl, by});
  tr->splits.push_back(d);
  tr->flops[tr->cur_stage] += fl;
  tr->bytes[tr->cur_stage] += by;
  return VP_OK;
}

// A slicing step (split precision): contiguous over a whole family, or a listed subset.
int add_slice(vp_tree_s* tr, int family, int buf, int K, int kseg, long long seg_stride, long long cstride,
              long long n, const std::vector<long long>* base, const std::vector<long long>* vid, cudaStream_t s) {
  DevSlice d{family, buf, K, kseg, seg_stride, cstride, n, nullptr, nullptr};
  int rc;
  long long* p = nullptr;
  if (base) { if ((rc = dev_upload(tr, *base, &p, s))) return rc; d.base = p; }
  if (vid) { if ((rc = dev_upload(tr, *vid, &p, s))) return rc; d.vid = p; }
  if (n <= 0) return VP_OK;
  const double by = (double)n * (8.0 * K + 2.0 * kSplitSlices * split_kpad(K) + 4.0);
  tr->steps.push_back({3, (int)tr->slice_ops.size(), tr->cur_stage, 0.0, by});
  tr->bytes[tr->cur_stage] += by;
  tr->slice_ops.push_back(d);
  return VP_OK;
}

int upload_reduce(vp_tree_s* tr, HostReduce& r, cudaStream_t s) {
  if (r.dst_off.empty()) return VP_OK;
  DevReduce d{};
  d.args.M = r.M; d.args.n = tr->T->n; d.args.final_out = r.final_out; d.args.N = tr->N;
  long long *a, *b, *c;
  int rc;
  if ((rc = dev_upload(tr, r.dst_off, &a, s))) return rc;
  if ((rc = dev_upload(tr, r.ptr, &b, s))) return rc;
  if ((rc = dev_upload(tr, r.slot, &c, s))) return rc;
  if (r.slot.empty()) {
    // a reduction with no contributions writes zeros; give it a valid (unused) slot array
    c = b;
  }
  d.args.dst_off = a; d.args.ptr = b; d.args.slot = c;
  d.dst = r.dst; d.src = r.src; d.n_dst = (int)r.dst_off.size();
  // in split precision every slot producer writes double-float slots
  const double fl = (double)r.M * (double)r.slot.size();
  const double by = 8.0 * (double)r.M * ((double)r.slot.size() + (double)r.dst_off.size());
  tr->steps.push_back({tr->T->precision == VP_PREC_SPLIT ? 5 : 1, (int)tr->reduces.size(), tr->cur_stage, fl, by});
  tr->flops[tr->cur_stage] += fl;
  tr->bytes[tr->cur_stage] += by;
  tr->reduces.push_back(d);
  return VP_OK;
}

const double* table_ptr(const vp_tables_s* T, int t) {
  switch (t) {
    case T_NEAR: return T->near;
    case T_S2M: return T->s2m;
    case T_L2T: return T->l2t;
    case T_M2M: return T->m2m;
    case T_L2L: return T->l2l;
    case T_M2L: return T->m2l;
    case T_M2T: return T->m2t;
    case T_S2L: return T->s2l;
  }
  return nullptr;
}

}  // namespace


int build_tree(vp_tree_s* tr, const TreePlan& P, cudaStream_t s) {
  const vp_tables_s* T = tr->T;
  const int n = T->n, C = T->C, E = T->E, nch = T->nch;
  const auto& B = P.boxes;
  const long long NB = (long long)B.size();
  auto kact = [&](int l) { return l >= 0 && l <= T->levels && T->kactive[l]; };

  // ---- local slots (M2L, S2L) and output slots (L2T, M2T, near)
  std::vector<std::vector<long long>> lsl((size_t)NB * nch);
  std::vector<std::vector<long long>> usl(B.size());
  long long nls = 0, nus = 0;
  HostGemm m2l, s2l, l2t, m2t, nearg, s2m;
  m2l.M = C; m2l.K = C; m2l.lda = C; m2l.table = T_M2L; m2l.src = BUF_MP; m2l.dst = BUF_LSLOT; m2l.split_vec = 1;
  for (const Pair& v : P.V) {
    const int l = B[v.tgt].level;
    for (int ch = 0; ch < nch; ++ch) {
      if (ch == 0 && !kact(l)) continue;
      const long long slot = nls++;
      lsl[(size_t)v.tgt * nch + ch].push_back(slot * C);
      m2l.entries.push_back({(long long)(l * T->m2l_stride_lvl() + v.pos * T->m2l_stride_off() + ch * T->m2l_stride_ch()),
                             (long long)v.src * E + ch * C, slot * C});
    }
  }
  s2l.M = C; s2l.K = n; s2l.lda = n; s2l.table = T_S2L; s2l.src = BUF_F; s2l.dst = BUF_LSLOT; s2l.split_vec = 0;
  for (const Pair& x : P.X) {
    const int l = B[x.tgt].level;
    for (int ch = 0; ch < nch; ++ch) {
      if (ch == 0 && !kact(l)) continue;
      const long long slot = nls++;
      lsl[(size_t)x.tgt * nch + ch].push_back(slot * C);
      s2l.entries.push_back({(long long)(l * T->s2l_stride_lvl() + x.pos * T->s2l_stride_pos() + ch * T->s2l_stride_ch()),
                             (long long)B[x.src].leaf * n, slot * C});
    }
  }
  nearg.M = 3 * n; nearg.K = n; nearg.lda = n; nearg.table = T_NEAR; nearg.src = BUF_F; nearg.dst = BUF_USLOT;
  nearg.split_vec = 0;
  for (const Pair& u : P.U) {
    const int l = B[u.tgt].level;
    const long long slot = nus++;
    usl[u.tgt].push_back(slot * 3 * n);
    nearg.entries.push_back({(long long)(l * T->near_stride_lvl() + u.pos * T->near_stride_pos()),
                             (long long)B[u.src].leaf * n, slot * 3 * n});
  }
  m2t.M = 3 * n; m2t.K = C; m2t.lda = C; m2t.table = T_M2T; m2t.src = BUF_MP; m2t.dst = BUF_USLOT; m2t.split_vec = 1;
  for (const Pair& w : P.W) {
    const int l = B[w.tgt].level;
    for (int ch = 0; ch < nch; ++ch) {
      if (ch == 0 && !kact(l + 1)) continue;
      const long long slot = nus++;
      usl[w.tgt].push_back(slot * 3 * n);
      m2t.entries.push_back({(long long)(l * T->m2t_stride_lvl() + w.pos * T->m2t_stride_pos() + ch * T->m2t_stride_ch()),
                             (long long)w.src * E + ch * C, slot * 3 * n});
    }
  }
  l2t.M = 3 * n; l2t.K = E; l2t.lda = E; l2t.table = T_L2T; l2t.src = BUF_LOC; l2t.dst = BUF_USLOT; l2t.split_vec = 2;
  s2m.M = E; s2m.K = n; s2m.lda = n; s2m.table = T_S2M; s2m.src = BUF_F; s2m.dst = BUF_MP; s2m.split_vec = 0;
  s2m.out_mode = 1;
  for (long long i = 0; i < NB; ++i) {
    const Box& b = B[i];
    if (b.leaf < 0 || b.level < 2) continue;
    const long long slot = nus++;
    usl[i].push_back(slot * 3 * n);
    l2t.entries.push_back({(long long)(b.level * T->l2t_stride_lvl()), i * E, slot * 3 * n});
    s2m.entries.push_back({(long long)(b.level * T->s2m_stride_lvl()), (long long)b.leaf * n, i * E});
  }
  tr->n_lslot = nls;
  tr->n_uslot = nus;

  // ---- device buffers
  TRY(cudaMalloc(&tr->mp, std::max<long long>(1, NB * E) * sizeof(double)));
  tr->allocs.push_back(tr->mp);
  TRY(cudaMalloc(&tr->loc, std::max<long long>(1, NB * E) * sizeof(double)));
  tr->allocs.push_back(tr->loc);
  TRY(cudaMalloc(&tr->lslot, std::max<long long>(1, nls * C) * sizeof(double)));
  tr->allocs.push_back(tr->lslot);
  TRY(cudaMalloc(&tr->uslot, std::max<long long>(1, nus * 3 * n) * sizeof(double)));
  tr->allocs.push_back(tr->uslot);
  const bool split = T->precision == VP_PREC_SPLIT;
  if (split) {
    // sliced source vectors of every family
    const long long nv[kVecFamilies] = {tr->n_leaves, NB * nch, NB, NB * nch, NB * nch, NB * nch};
    const int kk[kVecFamilies] = {n, C, E, 2 * C, C, 2 * C};
    for (int v = 0; v < kVecFamilies; ++v) {
      TRY(cudaMalloc(&tr->sv[v], std::max<long long>(1, nv[v] * kSplitSlices * split_kpad(kk[v])) * 2));
      tr->allocs.push_back(tr->sv[v]);
      TRY(cudaMalloc(&tr->se[v], std::max<long long>(1, nv[v]) * sizeof(int)));
      tr->allocs.push_back(tr->se[v]);
    }
  }

  int rc;
  // ---- steps, in pass order
  tr->cur_stage = VP_STAGE_UPWARD;
  tr->steps.push_back({2, 0, tr->cur_stage, 0.0, 8.0 * (double)NB * E});  // clear multipoles
  tr->bytes[tr->cur_stage] += 8.0 * (double)NB * E;
  if (split && (rc = add_slice(tr, 0, BUF_F, n, n, 0, n, tr->n_leaves, nullptr, nullptr, s))) return rc;
  if ((rc = upload_gemm(tr, s2m, s))) return rc;
  for (int l = P.max_level - 1; l >= 2; --l) {
    if (!split) {
      HostGemm m2m;
      m2m.M = C; m2m.K = 4 * C; m2m.kseg = C; m2m.seg_stride = E; m2m.lda = 4 * C; m2m.table = T_M2M;
      m2m.src = BUF_MP; m2m.dst = BUF_MP;
      for (long long i = 0; i < NB; ++i) {
        if (B[i].level != l || B[i].leaf >= 0) continue;
        for (int ch = 0; ch < nch; ++ch) {
          if (ch == 0 && !kact(l)) continue;
          m2m.entries.push_back({(long long)(l * T->m2m_stride_lvl() + ch * T->m2m_stride_ch()),
                                 (long long)B[i].child0 * E + ch * C, i * E + ch * C});
        }
      }
      if ((rc = upload_gemm(tr, m2m, s))) return rc;
      continue;
    }
    // split precision: children 0-1 (overwrite) then children 2-3 (accumulate), K = 2C each
    for (int half = 0; half < 2; ++half) {
      HostGemm m2m;
      m2m.M = C; m2m.K = 2 * C; m2m.kseg = C; m2m.seg_stride = E; m2m.lda = 4 * C;
      m2m.table = half ? T_M2M_HI : T_M2M_LO;
      m2m.src = BUF_MP; m2m.dst = BUF_MP; m2m.split_vec = half ? 5 : 3; m2m.out_mode = half ? 2 : 1;
      std::vector<long long> sbase, svid;
      for (long long i = 0; i < NB; ++i) {
        if (B[i].level != l || B[i].leaf >= 0) continue;
        for (int ch = 0; ch < nch; ++ch) {
          if (ch == 0 && !kact(l)) continue;
          const long long src = (long long)(B[i].child0 + 2 * half) * E + ch * C;
          m2m.entries.push_back({(long long)(l * T->m2m_stride_lvl() + ch * T->m2m_stride_ch()), src,
                                 i * E + ch * C, i * nch + ch});
          sbase.push_back(src);
          svid.push_back(i * nch + ch);
        }
      }
      if ((rc = add_slice(tr, half ? 5 : 3, BUF_MP, 2 * C, C, E, 0, (long long)svid.size(), &sbase, &svid, s)))
        return rc;
      if ((rc = upload_gemm(tr, m2m, s))) return rc;
    }
  }
  tr->cur_stage = VP_STAGE_M2L;
  if (split && (rc = add_slice(tr, 1, BUF_MP, C, C, 0, C, NB * nch, nullptr, nullptr, s))) return rc;
  if ((rc = upload_gemm(tr, m2l, s))) return rc;
  if ((rc = upload_gemm(tr, s2l, s))) return rc;
  tr->cur_stage = VP_STAGE_DOWNWARD;
  {
    HostReduce r;
    r.M = C; r.dst = BUF_LOC; r.src = BUF_LSLOT;
    r.ptr.push_back(0);
    for (long long i = 0; i < NB; ++i) {
      if (B[i].level < 2) continue;
      for (int ch = 0; ch < nch; ++ch) {
        r.dst_off.push_back(i * E + ch * C);
        for (long long o : lsl[(size_t)i * nch + ch]) r.slot.push_back(o);
        r.ptr.push_back((long long)r.slot.size());
      }
    }
    if ((rc = upload_reduce(tr, r, s))) return rc;
  }
  for (int l = 3; l <= P.max_level; ++l) {
    HostGemm l2l;
    l2l.M = C; l2l.K = C; l2l.lda = C; l2l.accumulate = 1; l2l.table = T_L2L; l2l.src = BUF_LOC; l2l.dst = BUF_LOC;
    l2l.split_vec = 4; l2l.out_mode = 2;
    std::vector<long long> sbase, svid;
    for (long long i = 0; i < NB; ++i) {
      if (B[i].level != l) continue;
      const int par = B[i].parent;
      const int q = (int)(i - B[par].child0);
      for (int ch = 0; ch < nch; ++ch) {
        if (ch == 0 && !kact(l - 1)) continue;
        l2l.entries.push_back({(long long)((l - 1) * T->l2l_stride_lvl() + q * T->l2l_stride_q() + ch * T->l2l_stride_ch()),
                               (long long)par * E + ch * C, i * E + ch * C, (long long)par * nch + ch});
        if (q == 0) {  // each parent's local is sliced once
          sbase.push_back((long long)par * E + ch * C);
          svid.push_back((long long)par * nch + ch);
        }
      }
    }
    if (split && (rc = add_slice(tr, 4, BUF_LOC, C, C, 0, 0, (long long)svid.size(), &sbase, &svid, s))) return rc;
    if ((rc = upload_gemm(tr, l2l, s))) return rc;
  }
  tr->cur_stage = VP_STAGE_TARGETS;
  if (split && (rc = add_slice(tr, 2, BUF_LOC, E, E, 0, E, NB, nullptr, nullptr, s))) return rc;
  if ((rc = upload_gemm(tr, l2t, s))) return rc;
  if ((rc = upload_gemm(tr, m2t, s))) return rc;
  tr->cur_stage = VP_STAGE_NEAR;
  if ((rc = upload_gemm(tr, nearg, s))) return rc;
  tr->cur_stage = VP_STAGE_OUTPUT;
  {
    HostReduce r;
    r.M = 3 * n; r.final_out = 1; r.src = BUF_USLOT;
    r.ptr.push_back(0);
    for (int k = 0; k < tr->n_leaves; ++k) {
      const int bi = P.leaf_box[k];
      r.dst_off.push_back((long long)k * n);
      for (long long o : usl[bi]) r.slot.push_back(o);
      r.ptr.push_back((long long)r.slot.size());
    }
    if ((rc = upload_reduce(tr, r, s))) return rc;
  }
  return VP_OK;
}

// ---------------------------------------------------------------------------------------------
// Layer-potential program (vp_layer_*): the double-layer velocity of boundary point sources at every
// node of the tree, both components, through the same grouped contractions as the volume
// potential. Boxes whose subtree holds no source carry no multipole and are left out of the
// upward pass and of the source side of the V and W lists; every box still receives locals and
// every leaf its values. Point-source operators (layer.cu) replace the leaf sources: multipoles
// of source leaves, locals of X-list targets, and direct values for adjacent (U-list) leaves.

// Sources binned by leaf box: sources perm[first[b] .. first[b] + count[b]) lie in box b.
struct LayerBins {
  std::vector<int> first, count;
  int max_ns = 0;
};

int upload_pt(vp_tree_s* tr, std::vector<PtInst>& inst, int rows, int rb, long long bs, int dst_buf, int kind,
              const PtSources& S, cudaStream_t s) {
  if (inst.empty()) return VP_OK;
  const vp_tables_s* T = tr->T;
  long long total = 0;
  int max_ns = 0;
  double fl = 0.0;
  for (PtInst& I : inst) {
    I.aoff = total;
    total += (long long)rows * 2 * I.ns;
    max_ns = std::max(max_ns, I.ns);
    fl += 2.0 * rows * 2.0 * I.ns;
  }
  DevPt d;
  d.n_inst = (int)inst.size(); d.rows = rows; d.rb = rb; d.bs = bs; d.dst = dst_buf;
  int rc;
  if ((rc = dev_upload(tr, inst, &d.inst, s))) return rc;
  void* A = nullptr;
  TRY(cudaMalloc(&A, (size_t)total * sizeof(double)));
  tr->allocs.push_back(A);
  d.A = static_cast<double*>(A);
  if (kind == 2) rc = launch_pt_near(T->alpha, T->p, tr->d_xi, d.inst, d.n_inst, max_ns, S, d.A, s);
  else rc = launch_pt_coeffs(kind, T->alpha, T->P, d.inst, d.n_inst, max_ns, S, d.A, s);
  if (rc) return rc;
  const double by = 8.0 * (double)total + 8.0 * (double)rows * (double)inst.size();
  tr->steps.push_back({6, (int)tr->pts.size(), tr->cur_stage, fl, by});
  tr->flops[tr->cur_stage] += fl;
  tr->bytes[tr->cur_stage] += by;
  tr->pts.push_back(d);
  return VP_OK;
}

int build_layer(vp_tree_s* tr, const TreePlan& P, const LayerBins& bins, const PtSources& S, cudaStream_t s) {
  const vp_tables_s* T = tr->T;
  const int n = T->n, C = T->C, E = T->E, nch = T->nch;
  constexpr int NC = 2;                  // velocity components
  const int Cs = (C + 1) & ~1, Us = (n + 1) & ~1;
  tr->lslot_stride = Cs;
  tr->uslot_stride = Us;
  const auto& B = P.boxes;
  const long long NB = (long long)B.size();
  auto kact = [&](int l) { return l >= 0 && l <= T->levels && T->kactive[l]; };
  auto off = [&](int a, long long b) { return (a * NB + b) * E; };  // coefficients of (component, box)
  const double x0 = tr->cx - 0.5 * T->side, y0 = tr->cy - 0.5 * T->side;
  // boxes whose subtree holds sources (children are numbered after their parent)
  std::vector<char> has(NB, 0);
  for (long long i = NB - 1; i >= 0; --i) {
    if (B[i].leaf >= 0) has[i] = bins.count[i] > 0;
    else
      for (int q = 0; q < 4; ++q) has[i] |= has[B[i].child0 + q];
  }
  std::vector<std::vector<long long>> lsl((size_t)NC * NB * nch), usl((size_t)NC * NB);
  long long nls = 0, nus = 0;

  std::vector<PtInst> ps2m, ps2l, pnear;
  for (long long i = 0; i < NB; ++i) {
    const Box& b = B[i];
    if (b.leaf < 0 || b.level < 2 || bins.count[i] == 0) continue;
    const double h = T->h(b.level), r = h / std::sqrt(2.0);
    PtInst I{};
    I.cx = x0 + (b.ix + 0.5) * h; I.cy = y0 + (b.iy + 0.5) * h; I.R = 1.25 * r; I.r = r;
    I.j0 = bins.first[i]; I.ns = bins.count[i]; I.kact = kact(b.level); I.dst = off(0, i);
    ps2m.push_back(I);
  }
  HostGemm m2l, l2t, m2t;
  m2l.M = C; m2l.K = C; m2l.lda = C; m2l.table = T_M2L; m2l.src = BUF_MP; m2l.dst = BUF_LSLOT; m2l.split_vec = 1;
  for (const Pair& v : P.V) {
    if (!has[v.src]) continue;
    const int l = B[v.tgt].level;
    for (int a = 0; a < NC; ++a)
      for (int ch = 0; ch < nch; ++ch) {
        if (ch == 0 && !kact(l)) continue;
        const long long slot = nls++;
        lsl[(size_t)(a * NB + v.tgt) * nch + ch].push_back(slot * Cs);
        m2l.entries.push_back({(long long)(l * T->m2l_stride_lvl() + v.pos * T->m2l_stride_off() + ch * T->m2l_stride_ch()),
                               off(a, v.src) + ch * C, slot * Cs});
      }
  }
  for (const Pair& x : P.X) {
    if (bins.count[x.src] == 0) continue;
    const Box& b = B[x.tgt];
    const double h = T->h(b.level), r = h / std::sqrt(2.0);
    const long long base = nls;
    nls += NC * nch;
    for (int a = 0; a < NC; ++a)
      for (int ch = 0; ch < nch; ++ch) lsl[(size_t)(a * NB + x.tgt) * nch + ch].push_back((base + a * nch + ch) * Cs);
    PtInst I{};
    I.cx = x0 + (b.ix + 0.5) * h; I.cy = y0 + (b.iy + 0.5) * h; I.R = r; I.r = r;
    I.j0 = bins.first[x.src]; I.ns = bins.count[x.src]; I.kact = kact(b.level); I.dst = base * Cs;
    ps2l.push_back(I);
  }
  l2t.M = n; l2t.K = E; l2t.lda = E; l2t.table = T_L2T; l2t.src = BUF_LOC; l2t.dst = BUF_USLOT; l2t.split_vec = 2;
  l2t.mat_elems = (long long)3 * n * E;  // values only: the leading n rows of the [3n x E] operator
  for (long long i = 0; i < NB; ++i) {
    const Box& b = B[i];
    if (b.leaf < 0 || b.level < 2) continue;
    for (int a = 0; a < NC; ++a) {
      const long long slot = nus++;
      usl[a * NB + i].push_back(slot * Us);
      l2t.entries.push_back({(long long)(b.level * T->l2t_stride_lvl()), off(a, i), slot * Us});
    }
  }
  m2t.M = n; m2t.K = C; m2t.lda = C; m2t.table = T_M2T; m2t.src = BUF_MP; m2t.dst = BUF_USLOT; m2t.split_vec = 1;
  m2t.mat_elems = (long long)3 * n * C;
  for (const Pair& w : P.W) {
    if (!has[w.src]) continue;
    const int l = B[w.tgt].level;
    for (int a = 0; a < NC; ++a)
      for (int ch = 0; ch < nch; ++ch) {
        if (ch == 0 && !kact(l + 1)) continue;
        const long long slot = nus++;
        usl[a * NB + w.tgt].push_back(slot * Us);
        m2t.entries.push_back({(long long)(l * T->m2t_stride_lvl() + w.pos * T->m2t_stride_pos() + ch * T->m2t_stride_ch()),
                               off(a, w.src) + ch * C, slot * Us});
      }
  }
  for (const Pair& u : P.U) {
    if (bins.count[u.src] == 0) continue;
    const Box& b = B[u.tgt];
    const double h = T->h(b.level);
    const long long base = nus;
    nus += NC;
    for (int a = 0; a < NC; ++a) usl[a * NB + u.tgt].push_back((base + a) * Us);
    PtInst I{};
    I.cx = x0 + b.ix * h; I.cy = y0 + b.iy * h; I.R = h; I.r = h;
    I.j0 = bins.first[u.src]; I.ns = bins.count[u.src]; I.kact = 1; I.dst = base * Us;
    pnear.push_back(I);
  }
  tr->n_lslot = nls;
  tr->n_uslot = nus;

  // ---- device buffers
  tr->mp_elems = NC * NB * E;
  TRY(cudaMalloc(&tr->mp, std::max<long long>(1, NC * NB * E) * sizeof(double)));
  tr->allocs.push_back(tr->mp);
  TRY(cudaMalloc(&tr->loc, std::max<long long>(1, NC * NB * E) * sizeof(double)));
  tr->allocs.push_back(tr->loc);
  TRY(cudaMalloc(&tr->lslot, std::max<long long>(1, nls * Cs) * sizeof(double)));
  tr->allocs.push_back(tr->lslot);
  TRY(cudaMalloc(&tr->uslot, std::max<long long>(1, nus * Us) * sizeof(double)));
  tr->allocs.push_back(tr->uslot);
  const bool split = T->precision == VP_PREC_SPLIT;
  if (split) {
    const long long nv[kVecFamilies] = {1, NC * NB * nch, NC * NB, NC * NB * nch, NC * NB * nch, NC * NB * nch};
    const int kk[kVecFamilies] = {n, C, E, 2 * C, C, 2 * C};
    for (int v = 0; v < kVecFamilies; ++v) {
      TRY(cudaMalloc(&tr->sv[v], std::max<long long>(1, nv[v] * kSplitSlices * split_kpad(kk[v])) * 2));
      tr->allocs.push_back(tr->sv[v]);
      TRY(cudaMalloc(&tr->se[v], std::max<long long>(1, nv[v]) * sizeof(int)));
      tr->allocs.push_back(tr->se[v]);
    }
  }

  int rc;
  tr->cur_stage = VP_STAGE_UPWARD;
  tr->steps.push_back({2, 0, tr->cur_stage, 0.0, 8.0 * (double)(NC * NB * E)});
  tr->bytes[tr->cur_stage] += 8.0 * (double)(NC * NB * E);
  if ((rc = upload_pt(tr, ps2m, 2 * E, E, NB * E, BUF_MP, 0, S, s))) return rc;
  for (int l = P.max_level - 1; l >= 2; --l) {
    if (!split) {
      HostGemm m2m;
      m2m.M = C; m2m.K = 4 * C; m2m.kseg = C; m2m.seg_stride = E; m2m.lda = 4 * C; m2m.table = T_M2M;
      m2m.src = BUF_MP; m2m.dst = BUF_MP;
      for (long long i = 0; i < NB; ++i) {
        if (B[i].level != l || B[i].leaf >= 0 || !has[i]) continue;
        for (int a = 0; a < NC; ++a)
          for (int ch = 0; ch < nch; ++ch) {
            if (ch == 0 && !kact(l)) continue;
            m2m.entries.push_back({(long long)(l * T->m2m_stride_lvl() + ch * T->m2m_stride_ch()),
                                   off(a, B[i].child0) + ch * C, off(a, i) + ch * C});
          }
      }
      if ((rc = upload_gemm(tr, m2m, s))) return rc;
      continue;
    }
    for (int half = 0; half < 2; ++half) {
      HostGemm m2m;
      m2m.M = C; m2m.K = 2 * C; m2m.kseg = C; m2m.seg_stride = E; m2m.lda = 4 * C;
      m2m.table = half ? T_M2M_HI : T_M2M_LO;
      m2m.src = BUF_MP; m2m.dst = BUF_MP; m2m.split_vec = half ? 5 : 3; m2m.out_mode = half ? 2 : 1;
      std::vector<long long> sbase, svid;
      for (long long i = 0; i < NB; ++i) {
        if (B[i].level != l || B[i].leaf >= 0 || !has[i]) continue;
        for (int a = 0; a < NC; ++a)
          for (int ch = 0; ch < nch; ++ch) {
            if (ch == 0 && !kact(l)) continue;
            const long long src = off(a, B[i].child0 + 2 * half) + ch * C;
            const long long vid = (a * NB + i) * nch + ch;
            m2m.entries.push_back({(long long)(l * T->m2m_stride_lvl() + ch * T->m2m_stride_ch()), src,
                                   off(a, i) + ch * C, vid});
            sbase.push_back(src);
            svid.push_back(vid);
          }
      }
      if ((rc = add_slice(tr, half ? 5 : 3, BUF_MP, 2 * C, C, E, 0, (long long)svid.size(), &sbase, &svid, s)))
        return rc;
      if ((rc = upload_gemm(tr, m2m, s))) return rc;
    }
  }
  tr->cur_stage = VP_STAGE_M2L;
  if (split && (rc = add_slice(tr, 1, BUF_MP, C, C, 0, C, NC * NB * nch, nullptr, nullptr, s))) return rc;
  if ((rc = upload_gemm(tr, m2l, s))) return rc;
  if ((rc = upload_pt(tr, ps2l, 2 * E, C, Cs, BUF_LSLOT, 1, S, s))) return rc;
  tr->cur_stage = VP_STAGE_DOWNWARD;
  {
    HostReduce r;
    r.M = C; r.dst = BUF_LOC; r.src = BUF_LSLOT;
    r.ptr.push_back(0);
    for (int a = 0; a < NC; ++a)
      for (long long i = 0; i < NB; ++i) {
        if (B[i].level < 2) continue;
        for (int ch = 0; ch < nch; ++ch) {
          r.dst_off.push_back(off(a, i) + ch * C);
          for (long long o : lsl[(size_t)(a * NB + i) * nch + ch]) r.slot.push_back(o);
          r.ptr.push_back((long long)r.slot.size());
        }
      }
    if ((rc = upload_reduce(tr, r, s))) return rc;
  }
  for (int l = 3; l <= P.max_level; ++l) {
    HostGemm l2l;
    l2l.M = C; l2l.K = C; l2l.lda = C; l2l.accumulate = 1; l2l.table = T_L2L; l2l.src = BUF_LOC; l2l.dst = BUF_LOC;
    l2l.split_vec = 4; l2l.out_mode = 2;
    std::vector<long long> sbase, svid;
    for (long long i = 0; i < NB; ++i) {
      if (B[i].level != l) continue;
      const int par = B[i].parent;
      const int q = (int)(i - B[par].child0);
      for (int a = 0; a < NC; ++a)
        for (int ch = 0; ch < nch; ++ch) {
          if (ch == 0 && !kact(l - 1)) continue;
          const long long vid = (a * NB + par) * nch + ch;
          l2l.entries.push_back({(long long)((l - 1) * T->l2l_stride_lvl() + q * T->l2l_stride_q() + ch * T->l2l_stride_ch()),
                                 off(a, par) + ch * C, off(a, i) + ch * C, vid});
          if (q == 0) {
            sbase.push_back(off(a, par) + ch * C);
            svid.push_back(vid);
          }
        }
    }
    if (split && (rc = add_slice(tr, 4, BUF_LOC, C, C, 0, 0, (long long)svid.size(), &sbase, &svid, s))) return rc;
    if ((rc = upload_gemm(tr, l2l, s))) return rc;
  }
  tr->cur_stage = VP_STAGE_TARGETS;
  if (split && (rc = add_slice(tr, 2, BUF_LOC, E, E, 0, E, NC * NB, nullptr, nullptr, s))) return rc;
  if ((rc = upload_gemm(tr, l2t, s))) return rc;
  if ((rc = upload_gemm(tr, m2t, s))) return rc;
  tr->cur_stage = VP_STAGE_NEAR;
  if ((rc = upload_pt(tr, pnear, 2 * n, n, Us, BUF_USLOT, 2, S, s))) return rc;
  tr->cur_stage = VP_STAGE_OUTPUT;
  {
    HostReduce r;
    r.M = n; r.final_out = 1; r.src = BUF_USLOT;
    r.ptr.push_back(0);
    for (int a = 0; a < NC; ++a)
      for (int k = 0; k < tr->n_leaves; ++k) {
        const int bi = P.leaf_box[k];
        r.dst_off.push_back(a * tr->N + (long long)k * n);
        for (long long o : usl[a * NB + bi]) r.slot.push_back(o);
        r.ptr.push_back((long long)r.slot.size());
      }
    if ((rc = upload_reduce(tr, r, s))) return rc;
  }
  return VP_OK;
}

// Kernel arguments of one split-precision launch with the engine set in d.
SplitArgs split_args(const vp_tree_s* tr, const DevSplit& d, double* const* bufs) {
  const SplitTables* stt = static_cast<const SplitTables*>(tr->T->near_split);
  const SplitTable* tb = d.table == T_NEAR ? &stt->near : d.table == T_S2M ? &stt->s2m : d.table == T_L2T
                         ? &stt->l2t : d.table == T_M2L ? &stt->m2l : d.table == T_M2T ? &stt->m2t
                         : d.table == T_M2M_LO ? &stt->m2m_lo : d.table == T_M2M_HI ? &stt->m2m_hi
                         : d.table == T_L2L ? &stt->l2l : &stt->s2l;
  SplitArgs a = d.args;
  a.A = static_cast<const slice_t*>(tb->A);
  a.ea = tb->ea;
  a.nrt = tb->nrt;
  a.ea_ld = tb->M;
  a.B = static_cast<const slice_t*>(tr->sv[d.vec]);
  a.eb = tr->se[d.vec];
  a.Y = bufs[d.dst];
  a.tiles = d.tiles[d.engine];
  return a;
}

// Issue one evaluation. With per-stage events (ev) every step goes to `s` in order. Otherwise the
// near-field steps, which need only the source (and its slices), run on `s` while the far-field
// chain (upward, M2L, downward, targets) runs on the tree's high-priority side stream; near-field
// CTAs then hold two tiles each, so chain launches find SMs; `s` waits for the chain before the
// output reduction. The two write disjoint contribution slots.
// With per-step events (step_ev, steps + 1 of them) every step goes to `s` in order and an event is
// recorded before each step and after the last.
int run_steps(vp_tree_s* tr, const double* f, double* u, double* g, cudaStream_t s0, cudaEvent_t* ev = nullptr,
              cudaEvent_t* step_ev = nullptr) {
  const vp_tables_s* T = tr->T;
  int stage = -1;
  const double* bufs_c[BUF_COUNT] = {f, tr->mp, tr->loc, tr->lslot, tr->uslot};
  double* bufs[BUF_COUNT] = {nullptr, tr->mp, tr->loc, tr->lslot, tr->uslot};
  const bool overlap = !ev && !step_ev && tr->side;
  int step_no = 0;
  bool src_ready = false, near_started = false, joined = !overlap;
  if (overlap) {
    TRY(cudaEventRecord(tr->ev_fork, s0));
    TRY(cudaStreamWaitEvent(tr->side, tr->ev_fork, 0));
  }
  for (const Step& st : tr->steps) {
    if (ev) {
      while (stage < st.stage) { ++stage; TRY(cudaEventRecord(ev[stage], s0)); }
    }
    if (step_ev) TRY(cudaEventRecord(step_ev[step_no], s0));
    ++step_no;
    const bool near_step = overlap && st.stage == VP_STAGE_NEAR;
    if (overlap && st.stage == VP_STAGE_OUTPUT && !joined) {
      TRY(cudaEventRecord(tr->ev_join, tr->side));
      TRY(cudaStreamWaitEvent(s0, tr->ev_join, 0));
      joined = true;
    }
    if (near_step && !near_started) {
      if (src_ready) TRY(cudaStreamWaitEvent(s0, tr->ev_src, 0));  // sliced source made on the chain
      near_started = true;
    }
    const cudaStream_t s = (!overlap || near_step || st.stage == VP_STAGE_OUTPUT) ? s0 : tr->side;
    if (st.kind == 2) {
      const long long elems = tr->mp_elems ? tr->mp_elems : (long long)tr->n_boxes * T->E;
      TRY(cudaMemsetAsync(tr->mp, 0, (size_t)elems * sizeof(double), s));
    } else if (st.kind == 0) {
      const DevGemm& d = tr->gemms[st.index];
      GemmArgs a = d.args;
      a.A = table_ptr(T, d.table);
      a.X = bufs_c[d.src];
      a.Y = bufs[d.dst];
      if (d.table == T_NEAR) k_gemm_gather_f64<1><<<d.n_tiles, 256, 0, s>>>(a);
      else k_gemm_gather_f64<0><<<d.n_tiles, 256, 0, s>>>(a);
      TRY(cudaGetLastError());
    } else if (st.kind == 1) {
      const DevReduce& d = tr->reduces[st.index];
      ReduceArgs a = d.args;
      a.S = bufs_c[d.src];
      if (a.final_out) { a.u = u; a.g = g; } else { a.Y = bufs[d.dst]; }
      const int threads = a.M >= 256 ? 256 : ((a.M + 31) / 32) * 32;
      if (a.M > 4 * threads) return VP_ERR_ARG;  // at most 4 rows per thread (3 p^2 <= 768)
      k_reduce<<<d.n_dst, threads, 0, s>>>(a);
      TRY(cudaGetLastError());
    } else if (st.kind == 7) {
      const DevNear& d = tr->nears[st.index];
      const int rc = launch_near_apply(d.n_nodes, d.node, d.ptr, d.panel, d.dW, bufs_c[BUF_F], tr->N, u, s);
      if (rc) return rc;
    } else if (st.kind == 6) {
      const DevPt& d = tr->pts[st.index];
      // slots of split-precision trees hold double-float values; multipole coefficients are FP64
      const int df = T->precision == VP_PREC_SPLIT && d.dst != BUF_MP;
      const int rc = launch_pt_apply(d.rows, d.rb, d.bs, df, d.inst, d.n_inst, tr->d_perm, bufs_c[BUF_F], d.A,
                                     bufs[d.dst], s);
      if (rc) return rc;
    } else if (st.kind == 3) {
      const DevSlice& d = tr->slice_ops[st.index];
      const int rc = launch_slice_list(bufs_c[d.buf], d.base, d.vid, d.n, d.K, d.kseg, d.seg_stride, d.cstride,
                                       tr->sv[d.family], tr->se[d.family], s);
      if (rc) return rc;
      if (overlap && d.family == 0 && !near_started) {
        TRY(cudaEventRecord(tr->ev_src, s));
        src_ready = true;
      }
    } else if (st.kind == 4) {
      const DevSplit& d = tr->splits[st.index];
      SplitArgs a = split_args(tr, d, bufs);
      const int rc = launch_split_gemm(a, d.n_tiles[d.engine], s, d.engine, near_step ? 1 : 0);
      if (rc) return rc;
    } else if (st.kind == 5) {
      const DevReduce& d = tr->reduces[st.index];
      DFReduceArgs a{};
      a.M = d.args.M; a.n = d.args.n; a.final_out = d.args.final_out; a.N = d.args.N;
      a.dst_off = d.args.dst_off; a.ptr = d.args.ptr; a.slot = d.args.slot;
      a.S = bufs_c[d.src];
      if (a.final_out) { a.u = u; a.g = g; } else { a.Y = bufs[d.dst]; }
      const int rc = launch_reduce_df(a, d.n_dst, s);
      if (rc) return rc;
    }
  }
  if (!joined) {
    TRY(cudaEventRecord(tr->ev_join, tr->side));
    TRY(cudaStreamWaitEvent(s0, tr->ev_join, 0));
  }
  if (step_ev) TRY(cudaEventRecord(step_ev[step_no], s0));
  if (ev) {
    while (stage < VP_NSTAGES) { ++stage; TRY(cudaEventRecord(ev[stage], s0)); }
  }
  return VP_OK;
}

}  // namespace vp

using namespace vp;

extern "C" int vp_tree_upload(vp_tables tables, double cx, double cy, int n_leaves, const int32_t* level,
                              const int32_t* ix, const int32_t* iy, void* stream, vp_tree* out) {
  if (!out) return VP_ERR_ARG;
  *out = nullptr;
  if (!tables || !level || !ix || !iy || n_leaves < 1 || !std::isfinite(cx) || !std::isfinite(cy)) return VP_ERR_ARG;
  TreePlan P;
  int rc = build_plan(n_leaves, level, ix, iy, tables->levels, P);
  if (rc != VP_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::unique_ptr<vp_tree_s> tr(new (std::nothrow) vp_tree_s());
  if (!tr) return VP_ERR_OOM;
  tr->T = tables;
  tr->n_leaves = n_leaves;
  tr->n_boxes = (int)P.boxes.size();
  tr->max_level = P.max_level;
  tr->N = (long long)n_leaves * tables->n;
  tr->cx = cx; tr->cy = cy;
  auto fail = [&](int code) { vp_tree_free(tr.release()); return code; };
  {
    std::vector<int> lv(level, level + n_leaves), xx(ix, ix + n_leaves), yy(iy, iy + n_leaves);
    tr->h_lv = lv; tr->h_ix = xx; tr->h_iy = yy;
    if ((rc = dev_upload(tr.get(), lv, &tr->d_lv, s))) return fail(rc);
    if ((rc = dev_upload(tr.get(), xx, &tr->d_ix, s))) return fail(rc);
    if ((rc = dev_upload(tr.get(), yy, &tr->d_iy, s))) return fail(rc);
    std::vector<double> xi(tables->p), w(tables->p);
    gauss_legendre_host(tables->p, xi.data(), w.data());
    if ((rc = dev_upload(tr.get(), xi, &tr->d_xi, s))) return fail(rc);
  }
  if ((rc = build_tree(tr.get(), P, s))) return fail(rc);
  {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&tr->side, cudaStreamNonBlocking, greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&tr->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&tr->ev_src, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&tr->ev_join, cudaEventDisableTiming) != cudaSuccess)
      return fail(VP_ERR_CUDA);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { set_last_cuda(e); return fail(VP_ERR_CUDA); }
  *out = tr.release();
  return VP_OK;
}

extern "C" int vp_tree_size(vp_tree tree, int64_t* n_leaves, int64_t* n_nodes) {
  if (!tree) return VP_ERR_ARG;
  if (n_leaves) *n_leaves = tree->n_leaves;
  if (n_nodes) *n_nodes = tree->N;
  return VP_OK;
}

extern "C" int vp_tree_nodes(vp_tree tree, double* xy, void* stream) {
  if (!tree || !xy) return VP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const vp_tables_s* T = tree->T;
  const long long N = tree->N;
  k_nodes<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(T->p, tree->n_leaves, tree->cx - 0.5 * T->side,
                                                     tree->cy - 0.5 * T->side, T->side, tree->d_lv, tree->d_ix,
                                                     tree->d_iy, tree->d_xi, N, xy);
  TRY(cudaGetLastError());
  return VP_OK;
}

extern "C" int vp_tree_interp(vp_tree tree, int n_fields, const double* fields, int n_points, const double* xy,
                              double* out, void* stream) {
  if (!tree || n_fields < 1 || n_points < 0 || (n_points > 0 && (!fields || !xy || !out))) return VP_ERR_ARG;
  if (n_points == 0) return VP_OK;
  if (tree->max_level > kInterpMaxLevel) return VP_ERR_LEVELS;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const vp_tables_s* T = tree->T;
  if (!tree->d_cell) {
    void* p = nullptr;
    const size_t cells = (size_t)1 << (2 * tree->max_level);
    TRY(cudaMalloc(&p, cells * sizeof(int)));
    tree->allocs.push_back(p);
    k_cell_map<<<tree->n_leaves, 256, 0, s>>>(tree->n_leaves, tree->max_level, tree->d_lv, tree->d_ix, tree->d_iy,
                                             static_cast<int*>(p));
    TRY(cudaGetLastError());
    tree->d_cell = static_cast<int*>(p);
  }
  k_interp<<<(unsigned)((n_points + 127) / 128), 128, 0, s>>>(
      T->p, tree->max_level, tree->cx - 0.5 * T->side, tree->cy - 0.5 * T->side, T->side, tree->d_lv, tree->d_ix,
      tree->d_iy, tree->d_xi, tree->d_cell, n_fields, fields, tree->N, n_points, xy, out);
  TRY(cudaGetLastError());
  return VP_OK;
}

extern "C" int vp_eval(vp_tree tree, const double* f, double* u, double* gradu, void* stream) {
  if (!tree || !f || !u || !gradu) return VP_ERR_ARG;
  return run_steps(tree, f, u, gradu, static_cast<cudaStream_t>(stream));
}

extern "C" int vp_eval_timed(vp_tree tree, const double* f, double* u, double* gradu, void* stream,
                             float* stage_ms) {
  if (!tree || !f || !u || !gradu || !stage_ms) return VP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t ev[VP_NSTAGES + 1];
  int made = 0;
  int rc = VP_OK;
  for (; made <= VP_NSTAGES; ++made) {
    if (cudaEventCreate(&ev[made]) != cudaSuccess) { rc = VP_ERR_CUDA; break; }
  }
  if (rc == VP_OK) rc = run_steps(tree, f, u, gradu, s, ev);
  if (rc == VP_OK) {
    cudaError_t e = cudaEventSynchronize(ev[VP_NSTAGES]);
    if (e != cudaSuccess) { set_last_cuda(e); rc = VP_ERR_CUDA; }
  }
  for (int k = 0; rc == VP_OK && k < VP_NSTAGES; ++k) {
    if (cudaEventElapsedTime(&stage_ms[k], ev[k], ev[k + 1]) != cudaSuccess) rc = VP_ERR_CUDA;
  }
  for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
  return rc;
}

extern "C" int vp_tree_bytes(vp_tree tree, double* stage_bytes) {
  if (!tree || !stage_bytes) return VP_ERR_ARG;
  for (int k = 0; k < VP_NSTAGES; ++k) stage_bytes[k] = tree->bytes[k];
  return VP_OK;
}

extern "C" int vp_eval_steps(vp_tree tree, const double* f, double* u, double* gradu, void* stream, int cap,
                             int* n_steps, float* ms, int* info, double* flops, double* bytes) {
  if (!tree || !n_steps) return VP_ERR_ARG;
  const int n = (int)tree->steps.size();
  *n_steps = n;
  if (cap <= 0) return VP_OK;
  if (cap < n || !f || !u || !gradu || !ms || !info || !flops || !bytes) return VP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<cudaEvent_t> ev(n + 1, nullptr);
  int rc = VP_OK;
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) { rc = VP_ERR_CUDA; break; }
  if (rc == VP_OK) rc = run_steps(tree, f, u, gradu, s, nullptr, ev.data());
  if (rc == VP_OK) {
    const cudaError_t e = cudaEventSynchronize(ev[n]);
    if (e != cudaSuccess) { set_last_cuda(e); rc = VP_ERR_CUDA; }
  }
  for (int k = 0; rc == VP_OK && k < n; ++k) {
    if (cudaEventElapsedTime(&ms[k], ev[k], ev[k + 1]) != cudaSuccess) { rc = VP_ERR_CUDA; break; }
    const Step& st = tree->steps[k];
    int table = -1, engine = -1;
    if (st.kind == 0) table = tree->gemms[st.index].table;
    if (st.kind == 4) { table = tree->splits[st.index].table; engine = tree->splits[st.index].engine; }
    info[4 * k] = st.kind; info[4 * k + 1] = st.stage; info[4 * k + 2] = table; info[4 * k + 3] = engine;
    flops[k] = st.flops;
    bytes[k] = st.bytes;
  }
  for (auto e : ev) if (e) cudaEventDestroy(e);
  return rc;
}

extern "C" int vp_tree_stats(vp_tree tree, int64_t* launches, double* stage_flops) {
  if (!tree) return VP_ERR_ARG;
  if (launches) {
    int64_t c = 0;
    for (const Step& st : tree->steps) { (void)st; ++c; }
    *launches = c;
  }
  if (stage_flops)
    for (int k = 0; k < VP_NSTAGES; ++k) stage_flops[k] = tree->flops[k];
  return VP_OK;
}

namespace {
// Device address of page-locked host memory (cudaHostAlloc / cudaHostRegister), or null for any
// other pointer.
const void* mapped_host(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}
}  // namespace

extern "C" int vp_eval_host(vp_tree tree, const double* f, double* u, double* gradu, void* stream) {
  if (!tree || !f || !u || !gradu) return VP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t N = (size_t)tree->N;
  // Page-locked host buffers are used in place: the output reduction writes u and grad u straight
  // into them, and in the split form (where only the slicing kernel reads f) f is read from the
  // host as well. Other buffers go through device copies.
  const void* fm = tree->T->precision == VP_PREC_SPLIT ? mapped_host(f) : nullptr;
  void* um = const_cast<void*>(mapped_host(u));
  void* gm = const_cast<void*>(mapped_host(gradu));
  if (!tree->d_f && (!fm || !um || !gm)) {
    TRY(cudaMalloc(&tree->d_f, N * sizeof(double)));
    tree->allocs.push_back(tree->d_f);
    TRY(cudaMalloc(&tree->d_u, 3 * N * sizeof(double)));
    tree->allocs.push_back(tree->d_u);
    tree->d_g = tree->d_u + N;
  }
  const double* fd = static_cast<const double*>(fm);
  if (!fd) {
    TRY(cudaMemcpyAsync(tree->d_f, f, N * sizeof(double), cudaMemcpyHostToDevice, s));
    fd = tree->d_f;
  }
  double* ud = um && gm ? static_cast<double*>(um) : tree->d_u;
  double* gd = um && gm ? static_cast<double*>(gm) : tree->d_g;
  const int rc = run_steps(tree, fd, ud, gd, s);
  if (rc) return rc;
  if (ud == tree->d_u) {
    TRY(cudaMemcpyAsync(u, tree->d_u, N * sizeof(double), cudaMemcpyDeviceToHost, s));
    TRY(cudaMemcpyAsync(gradu, tree->d_g, 2 * N * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  TRY(cudaStreamSynchronize(s));
  return VP_OK;
}

extern "C" void vp_tree_free(vp_tree tree) {
  if (!tree) return;
  if (tree->side) cudaStreamDestroy(tree->side);
  for (cudaEvent_t e : {tree->ev_fork, tree->ev_src, tree->ev_join})
    if (e) cudaEventDestroy(e);
  for (void* p : tree->allocs) cudaFree(p);
  delete tree;
}

extern "C" const char* vp_last_cuda_error(void) { return cudaGetErrorString(last_cuda()); }

extern "C" const char* vp_strerror(int code) {
  switch (code) {
    case VP_OK: return "ok";
    case VP_ERR_ARG: return "invalid argument";
    case VP_ERR_TREE_UNBALANCED: return "adjacent leaves differ by more than one level";
    case VP_ERR_LEVELS: return "a leaf is deeper than the tables";
    case VP_ERR_OOM: return "out of memory";
    case VP_ERR_CUDA: return "CUDA runtime error";
    case VP_ERR_TREE: return "leaves overlap, leave gaps or lie outside the root box";
    case VP_ERR_TIMEOUT: return "a bounded device wait ran out";
  }
  return "unknown error";
}

// ---------------------------------------------------------------------------
// Engine selection and autotuning of the split-precision contractions.

extern "C" int vp_tree_set_engine(vp_tree tree, int engine) {
  if (!tree || engine < 0 || engine >= kEngines) return VP_ERR_ARG;
  for (auto& d : tree->splits) d.engine = engine;
  return VP_OK;
}

extern "C" int vp_selftest_timeout(void* stream) {
  const int rc = selftest_wait(2000000ll, static_cast<cudaStream_t>(stream));  // about a millisecond
  if (rc) return rc;
  return vp_device_status();
}

extern "C" int vp_device_status(void) {
  int flag = 0;
  const int rc = read_split_error(&flag);
  if (rc) return rc;
  return flag ? VP_ERR_TIMEOUT : VP_OK;
}

namespace vp {
namespace {

// Time every split-precision launch of one evaluation with the given engine (ms per launch).
int time_split_launches(vp_tree_s* tr, const double* f, double* u, double* g, int engine, cudaStream_t s,
                        std::vector<float>& ms) {
  for (auto& d : tr->splits) d.engine = engine;
  const int ns = (int)tr->splits.size();
  std::vector<cudaEvent_t> ev(2 * ns, nullptr);
  for (auto& x : ev) if (cudaEventCreate(&x) != cudaSuccess) return VP_ERR_CUDA;
  int rc = run_steps(tr, f, u, g, s);  // warm up
  double* bufs[BUF_COUNT] = {nullptr, tr->mp, tr->loc, tr->lslot, tr->uslot};
  for (int k = 0; rc == VP_OK && k < ns; ++k) {
    DevSplit d = tr->splits[k];
    d.engine = engine;
    SplitArgs a = split_args(tr, d, bufs);
    // accumulating outputs are only timed (their values are rebuilt by the next full evaluation)
    if (cudaEventRecord(ev[2 * k], s) != cudaSuccess) rc = VP_ERR_CUDA;
    if (rc == VP_OK) rc = launch_split_gemm(a, d.n_tiles[engine], s, engine);
    if (rc == VP_OK && cudaEventRecord(ev[2 * k + 1], s) != cudaSuccess) rc = VP_ERR_CUDA;
  }
  if (rc == VP_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = VP_ERR_CUDA;
  ms.assign(ns, 0.f);
  for (int k = 0; rc == VP_OK && k < ns; ++k)
    if (cudaEventElapsedTime(&ms[k], ev[2 * k], ev[2 * k + 1]) != cudaSuccess) rc = VP_ERR_CUDA;
  for (auto x : ev) if (x) cudaEventDestroy(x);
  return rc;
}

}  // namespace
}  // namespace vp

extern "C" int vp_autotune(vp_tree tree, const double* f, double* u, double* gradu, const char* cache_path,
                           void* stream, int* n_tcgen05) {
  if (!tree || !f || !u || !gradu) return VP_ERR_ARG;
  if (tree->T->precision != VP_PREC_SPLIT || tree->splits.empty()) {
    if (n_tcgen05) *n_tcgen05 = 0;
    return VP_OK;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int ns = (int)tree->splits.size();
  std::vector<int> choice(ns, -1);
  // cache: one line per launch "key engine", key = p P nch table M Kpad tiles
  auto key_of = [&](const DevSplit& d) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "%d %d %d %d %d %d %d", tree->T->p, tree->T->P, tree->T->nch, d.table,
                  d.args.M, d.args.Kpad, d.n_tiles[0]);
    return std::string(buf);
  };
  std::vector<std::pair<std::string, int>> cache;
  if (cache_path) {
    if (FILE* fp = std::fopen(cache_path, "r")) {
      char line[256];
      while (std::fgets(line, sizeof(line), fp)) {
        int a[7], eng;
        if (std::sscanf(line, "%d %d %d %d %d %d %d %d", &a[0], &a[1], &a[2], &a[3], &a[4], &a[5], &a[6], &eng) == 8) {
          char k[160];
          std::snprintf(k, sizeof(k), "%d %d %d %d %d %d %d", a[0], a[1], a[2], a[3], a[4], a[5], a[6]);
          cache.emplace_back(k, eng);
        }
      }
      std::fclose(fp);
    }
  }
  bool need = false;
  for (int k = 0; k < ns; ++k) {
    const std::string key = key_of(tree->splits[k]);
    for (auto& c : cache) if (c.first == key) choice[k] = c.second;
    if (choice[k] < 0) need = true;
  }
  if (need) {
    std::vector<float> tt[kEngines];
    int rc = VP_OK;
    for (int en = 0; en < kEngines && rc == VP_OK; ++en) rc = time_split_launches(tree, f, u, gradu, en, s, tt[en]);
    if (rc == VP_OK) rc = vp_device_status();
    if (rc != VP_OK) {
      vp_tree_set_engine(tree, kEngineMmaSync);
      return rc;
    }
    // one decision per key: the engine (tile shape) with the smallest total time over the launches
    // sharing it
    for (int k = 0; k < ns; ++k) {
      if (choice[k] >= 0) continue;
      const std::string key = key_of(tree->splits[k]);
      double tot[kEngines] = {};
      for (int m = 0; m < ns; ++m)
        if (key_of(tree->splits[m]) == key)
          for (int en = 0; en < kEngines; ++en) tot[en] += tt[en][m];
      int c = 0;
      for (int en = 1; en < kEngines; ++en)
        if (tot[en] < tot[c]) c = en;
      for (int m = 0; m < ns; ++m)
        if (choice[m] < 0 && key_of(tree->splits[m]) == key) choice[m] = c;
    }
    if (cache_path) {
      if (FILE* fp = std::fopen(cache_path, "a")) {
        for (int k = 0; k < ns; ++k) {
          bool cached = false;
          const std::string key = key_of(tree->splits[k]);
          for (auto& c : cache) cached |= (c.first == key);
          if (!cached) {
            std::fprintf(fp, "%s %d\n", key.c_str(), choice[k]);
            cache.emplace_back(key, choice[k]);
          }
        }
        std::fclose(fp);
      }
    }
  }
  int ntc = 0;
  for (int k = 0; k < ns; ++k) {
    tree->splits[k].engine = choice[k];
    ntc += choice[k] == kEngineTcgen05 || choice[k] == kEngineTcgen05N64 || choice[k] == kEngineTcgen05T;
  }
  if (n_tcgen05) *n_tcgen05 = ntc;
  // leave u, gradu holding a valid evaluation with the chosen engines
  return run_steps(tree, f, u, gradu, s);
}

// ---------------------------------------------------------------------------
// Batches: many independent trees (any kernel, alpha, p, depth) evaluated by one CUDA graph. Every
// tree's evaluation is a chain of launches on private work buffers, so the graph holds one branch
// per tree (captured on forked streams) and the hardware overlaps the branches; replaying the graph
// costs one launch from the host.
struct vp_batch_s {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int n_trees = 0;
  long long nodes = 0;
  int launches = 0;
};

namespace vp {
namespace {

int capture_trees(int n, const vp_tree* trees, const double* const* f, double* const* u, double* const* g,
                  int n_streams, cudaStream_t user, vp_batch_s* B) {
  std::vector<cudaStream_t> ss(n_streams, nullptr);
  std::vector<cudaEvent_t> ev(n_streams + 1, nullptr);
  int rc = VP_OK;
  // capture on a private stream (the legacy default stream cannot be captured); it first waits for
  // the caller's stream so that setup work queued there is complete
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return VP_ERR_CUDA;
  if (cudaStreamSynchronize(user) != cudaSuccess) { cudaStreamDestroy(s); return VP_ERR_CUDA; }
  for (int k = 0; k < n_streams && rc == VP_OK; ++k)
    if (cudaStreamCreateWithFlags(&ss[k], cudaStreamNonBlocking) != cudaSuccess) rc = VP_ERR_CUDA;
  for (int k = 0; k <= n_streams && rc == VP_OK; ++k)
    if (cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) != cudaSuccess) rc = VP_ERR_CUDA;
  bool capturing = false;
  if (rc == VP_OK) {
    const cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { set_last_cuda(e); rc = VP_ERR_CUDA; }
    else capturing = true;
  }
  if (rc == VP_OK && cudaEventRecord(ev[n_streams], s) != cudaSuccess) rc = VP_ERR_CUDA;
  for (int k = 0; k < n_streams && rc == VP_OK; ++k)
    if (cudaStreamWaitEvent(ss[k], ev[n_streams], 0) != cudaSuccess) rc = VP_ERR_CUDA;
  for (int t = 0; t < n && rc == VP_OK; ++t) {
    rc = run_steps(trees[t], f[t], u[t], g[t], ss[t % n_streams]);
    B->launches += (int)trees[t]->steps.size();
  }
  for (int k = 0; k < n_streams && rc == VP_OK; ++k) {
    if (cudaEventRecord(ev[k], ss[k]) != cudaSuccess || cudaStreamWaitEvent(s, ev[k], 0) != cudaSuccess)
      rc = VP_ERR_CUDA;
  }
  if (capturing) {
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (rc == VP_OK && e != cudaSuccess) { set_last_cuda(e); rc = VP_ERR_CUDA; }
    if (rc == VP_OK) B->graph = graph;
    else if (graph) cudaGraphDestroy(graph);
  }
  if (rc == VP_OK) {
    const cudaError_t e = cudaGraphInstantiate(&B->exec, B->graph, 0);
    if (e != cudaSuccess) { set_last_cuda(e); rc = VP_ERR_CUDA; }
  }
  for (auto x : ev) if (x) cudaEventDestroy(x);
  for (auto x : ss) if (x) cudaStreamDestroy(x);
  cudaStreamDestroy(s);
  return rc;
}

}  // namespace
}  // namespace vp

extern "C" int vp_batch_create(int n_trees, const vp_tree* trees, const double* const* f, double* const* u,
                               double* const* gradu, int n_streams, void* stream, vp_batch* out) {
  if (!out) return VP_ERR_ARG;
  *out = nullptr;
  if (n_trees < 1 || !trees || !f || !u || !gradu) return VP_ERR_ARG;
  for (int t = 0; t < n_trees; ++t)
    if (!trees[t] || !f[t] || !u[t] || !gradu[t]) return VP_ERR_ARG;
  if (n_streams < 1) n_streams = 1;
  if (n_streams > n_trees) n_streams = n_trees;
  if (n_streams > 128) n_streams = 128;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // per-device kernel attributes are set outside the capture
  for (int t = 0; t < n_trees; ++t)
    if (trees[t]->T->precision == VP_PREC_SPLIT) {
      const int rc = prepare_split_launch();
      if (rc) return rc;
      break;
    }
  std::unique_ptr<vp_batch_s> B(new (std::nothrow) vp_batch_s());
  if (!B) return VP_ERR_OOM;
  B->n_trees = n_trees;
  for (int t = 0; t < n_trees; ++t) B->nodes += trees[t]->N;
  const int rc = capture_trees(n_trees, trees, f, u, gradu, n_streams, s, B.get());
  if (rc != VP_OK) { vp_batch_free(B.release()); return rc; }
  *out = B.release();
  return VP_OK;
}

extern "C" int vp_batch_run(vp_batch batch, void* stream) {
  if (!batch || !batch->exec) return VP_ERR_ARG;
  const cudaError_t e = cudaGraphLaunch(batch->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) { set_last_cuda(e); return VP_ERR_CUDA; }
  return VP_OK;
}

extern "C" int vp_batch_stats(vp_batch batch, int64_t* nodes, int64_t* launches) {
  if (!batch) return VP_ERR_ARG;
  if (nodes) *nodes = batch->nodes;
  if (launches) *launches = batch->launches;
  return VP_OK;
}

extern "C" void vp_batch_free(vp_batch batch) {
  if (!batch) return;
  if (batch->exec) cudaGraphExecDestroy(batch->exec);
  if (batch->graph) cudaGraphDestroy(batch->graph);
  delete batch;
}

extern "C" int vp_eval_batched(int n_trees, const vp_tree* trees, const double* const* f, double* const* u,
                               double* const* gradu, int use_graph, void* stream) {
  if (n_trees < 1 || !trees || !f || !u || !gradu) return VP_ERR_ARG;
  if (use_graph) {
    vp_batch b = nullptr;
    int rc = vp_batch_create(n_trees, trees, f, u, gradu, 16, stream, &b);
    if (rc == VP_OK) rc = vp_batch_run(b, stream);
    if (rc == VP_OK) {
      const cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
      if (e != cudaSuccess) { set_last_cuda(e); rc = VP_ERR_CUDA; }
    }
    vp_batch_free(b);
    return rc;
  }
  for (int t = 0; t < n_trees; ++t) {
    if (!trees[t]) return VP_ERR_ARG;
    const int rc = run_steps(trees[t], f[t], u[t], gradu[t], static_cast<cudaStream_t>(stream));
    if (rc) return rc;
  }
  return VP_OK;
}

// ---------------------------------------------------------------------------
// Layer potential at the nodes of a tree (vp_layer_*).
struct vp_layer_s {
  vp_tree_s* prog = nullptr;  // the step program over the tree's boxes (owns its buffers)
  int n_src = 0;
  std::vector<double> src;                 // host copy of the points [5][n_src]
  std::vector<int> lv, ix, iy;             // the tree's leaves
  int p = 0;
  double cx = 0.0, cy = 0.0, side = 0.0;
  bool corrected = false;
};

extern "C" int vp_layer_create(vp_tree tree, int n_src, const double* src, void* stream, vp_layer* out) {
  if (!out) return VP_ERR_ARG;
  *out = nullptr;
  if (!tree || n_src < 1 || !src) return VP_ERR_ARG;
  vp_tables_s* T = tree->T;
  if (T->nch != 2) return VP_ERR_ARG;  // the double layer needs the two-channel (modified-biharmonic) bases
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TreePlan P;
  int rc = build_plan(tree->n_leaves, tree->h_lv.data(), tree->h_ix.data(), tree->h_iy.data(), T->levels, P);
  if (rc != VP_OK) return rc;
  const auto& B = P.boxes;
  const long long NB = (long long)B.size();
  // bin the sources by leaf box (descending from the root; a point on a box edge goes to the child
  // above / to the right)
  const double x0 = tree->cx - 0.5 * T->side, y0 = tree->cy - 0.5 * T->side;
  std::vector<int> box_of(n_src);
  for (int j = 0; j < n_src; ++j) {
    const double x = src[j], y = src[n_src + j];
    if (!std::isfinite(x) || !std::isfinite(y) || x < x0 || y < y0 || x > x0 + T->side || y > y0 + T->side)
      return VP_ERR_ARG;
    const double w = src[4 * (size_t)n_src + j];
    if (!std::isfinite(w) || !std::isfinite(src[2 * (size_t)n_src + j]) || !std::isfinite(src[3 * (size_t)n_src + j]))
      return VP_ERR_ARG;
    int b = 0;
    while (B[b].leaf < 0) {
      const double h = T->h(B[b].level);
      const double cx = x0 + (B[b].ix + 0.5) * h, cy = y0 + (B[b].iy + 0.5) * h;
      b = B[b].child0 + (x >= cx ? 1 : 0) + (y >= cy ? 2 : 0);
    }
    box_of[j] = b;
  }
  LayerBins bins;
  bins.first.assign(NB, 0);
  bins.count.assign(NB, 0);
  for (int j = 0; j < n_src; ++j) ++bins.count[box_of[j]];
  {
    int acc = 0;
    for (long long b = 0; b < NB; ++b) { bins.first[b] = acc; acc += bins.count[b]; bins.max_ns = std::max(bins.max_ns, bins.count[b]); }
  }
  std::vector<int> perm(n_src), fill(bins.first);
  for (int j = 0; j < n_src; ++j) perm[fill[box_of[j]]++] = j;

  std::unique_ptr<vp_tree_s> pr(new (std::nothrow) vp_tree_s());
  if (!pr) return VP_ERR_OOM;
  pr->T = T;
  pr->n_leaves = tree->n_leaves;
  pr->n_boxes = (int)NB;
  pr->max_level = P.max_level;
  pr->N = tree->N;
  pr->cx = tree->cx; pr->cy = tree->cy;
  auto fail = [&](int code) { vp_tree_free(pr.release()); return code; };
  {
    std::vector<double> xi(T->p), w(T->p);
    gauss_legendre_host(T->p, xi.data(), w.data());
    if ((rc = dev_upload(pr.get(), xi, &pr->d_xi, s))) return fail(rc);
  }
  std::vector<double> sv(src, src + 5 * (size_t)n_src);
  double* d_src = nullptr;
  if ((rc = dev_upload(pr.get(), sv, &d_src, s))) return fail(rc);
  if ((rc = dev_upload(pr.get(), perm, &pr->d_perm, s))) return fail(rc);
  PtSources S{d_src, d_src + n_src, d_src + 2 * (size_t)n_src, d_src + 3 * (size_t)n_src, d_src + 4 * (size_t)n_src,
              pr->d_perm};
  if ((rc = build_layer(pr.get(), P, bins, S, s))) return fail(rc);
  {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&pr->side, cudaStreamNonBlocking, greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&pr->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pr->ev_src, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pr->ev_join, cudaEventDisableTiming) != cudaSuccess)
      return fail(VP_ERR_CUDA);
  }
  const cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { set_last_cuda(e); return fail(VP_ERR_CUDA); }
  std::unique_ptr<vp_layer_s> L(new (std::nothrow) vp_layer_s());
  if (!L) return fail(VP_ERR_OOM);
  L->prog = pr.release();
  L->n_src = n_src;
  L->src.assign(src, src + 5 * (size_t)n_src);
  L->lv = tree->h_lv; L->ix = tree->h_ix; L->iy = tree->h_iy;
  L->p = T->p; L->cx = tree->cx; L->cy = tree->cy; L->side = T->side;
  *out = L.release();
  return VP_OK;
}

namespace {
// Point and derivative of the star r(t) = R + A cos(k t + phase) (host).
void star_host(const StarGeom& g, double t, double& x, double& y, double& dx, double& dy) {
  const double c = std::cos(t), s = std::sin(t);
  const double r = g.R + g.A * std::cos(g.k * t + g.phase), dr = -g.A * g.k * std::sin(g.k * t + g.phase);
  x = r * c; y = r * s;
  dx = dr * c - r * s; dy = dr * s + r * c;
}
}  // namespace

extern "C" int vp_layer_near_star(vp_layer layer, double R, double A, int k, double phase, int n_panels,
                                  double dist, void* stream, int64_t* n_pairs_out) {
  if (!layer || !(R > 0.0) || !(A >= 0.0) || A >= R || k < 0 || n_panels < 1 || !(dist > 0.0) || dist > 8.0)
    return VP_ERR_ARG;
  if (layer->corrected) return VP_ERR_ARG;  // one correction per layer
  constexpr int Q = kNearQ;
  if ((long long)n_panels * Q != layer->n_src) return VP_ERR_ARG;
  const StarGeom g{R, A, phase, k, n_panels};
  const double hp = 2.0 * kPi / n_panels;
  std::vector<double> gx(Q), gw(Q);
  gauss_legendre_host(Q, gx.data(), gw.data());
  // the layer's points must be the star's panel nodes, in panel order
  const int n = layer->n_src;
  const double* S = layer->src.data();
  std::vector<double> plen(n_panels, 0.0);
  for (int pnl = 0; pnl < n_panels; ++pnl)
    for (int q = 0; q < Q; ++q) {
      const int j = pnl * Q + q;
      double x, y, dx, dy;
      star_host(g, pnl * hp + 0.5 * hp * (1.0 + gx[q]), x, y, dx, dy);
      const double sp = std::hypot(dx, dy);
      if (std::fabs(S[j] - x) > 1e-12 * (R + A) || std::fabs(S[n + j] - y) > 1e-12 * (R + A) ||
          std::fabs(S[2 * n + j] + dy / sp) > 1e-10 || std::fabs(S[3 * n + j] - dx / sp) > 1e-10)
        return VP_ERR_ARG;
      plen[pnl] += S[4 * n + j];
    }
  // node coordinates of the tree (host) and the pairs within dist panel lengths of a panel
  const int p = layer->p, nn = p * p;
  std::vector<double> xi(p), wi(p);
  gauss_legendre_host(p, xi.data(), wi.data());
  const double x0 = layer->cx - 0.5 * layer->side, y0 = layer->cy - 0.5 * layer->side;
  const int nl = (int)layer->lv.size();
  struct HP { long long node; int panel; double t0, d, x, y; };
  std::vector<HP> hp_pairs;
  constexpr int kSamp = 64;
  for (int pnl = 0; pnl < n_panels; ++pnl) {
    const double ta = pnl * hp, reach = dist * plen[pnl];
    double bx0 = 1e300, bx1 = -1e300, by0 = 1e300, by1 = -1e300;
    std::vector<double> sx(kSamp + 1), sy(kSamp + 1);
    for (int m = 0; m <= kSamp; ++m) {
      double dx, dy;
      star_host(g, ta + hp * m / kSamp, sx[m], sy[m], dx, dy);
      bx0 = std::min(bx0, sx[m]); bx1 = std::max(bx1, sx[m]);
      by0 = std::min(by0, sy[m]); by1 = std::max(by1, sy[m]);
    }
    bx0 -= reach; bx1 += reach; by0 -= reach; by1 += reach;
    for (int lf = 0; lf < nl; ++lf) {
      const double h = layer->side / (double)(1ll << layer->lv[lf]);
      const double lx = x0 + layer->ix[lf] * h, ly = y0 + layer->iy[lf] * h;
      if (lx > bx1 || lx + h < bx0 || ly > by1 || ly + h < by0) continue;
      for (int t = 0; t < nn; ++t) {
        const double x = lx + 0.5 * (1.0 + xi[t % p]) * h, y = ly + 0.5 * (1.0 + xi[t / p]) * h;
        if (x < bx0 || x > bx1 || y < by0 || y > by1) continue;
        int mb = 0;
        double best = 1e300;
        for (int m = 0; m <= kSamp; ++m) {
          const double d2 = (sx[m] - x) * (sx[m] - x) + (sy[m] - y) * (sy[m] - y);
          if (d2 < best) { best = d2; mb = m; }
        }
        // Newton on (y(t) - x) . y'(t) = 0 from the nearest sample, kept inside the panel
        double t0 = ta + hp * mb / kSamp;
        for (int it = 0; it < 30; ++it) {
          const double e = 1e-7 * hp;
          double yx, yy, dx, dy, ya, yb, dxa, dya;
          star_host(g, t0, yx, yy, dx, dy);
          const double f0 = (yx - x) * dx + (yy - y) * dy;
          star_host(g, t0 + e, ya, yb, dxa, dya);
          const double f1 = (ya - x) * dxa + (yb - y) * dya;
          const double fp = (f1 - f0) / e;
          if (!(fp > 0.0)) break;
          const double tn = std::min(ta + hp, std::max(ta, t0 - f0 / fp));
          const bool done = std::fabs(tn - t0) < 1e-15 * hp;
          t0 = tn;
          if (done) break;
        }
        double yx, yy, dx, dy;
        star_host(g, t0, yx, yy, dx, dy);
        const double d = std::hypot(yx - x, yy - y);
        if (d < reach) hp_pairs.push_back({(long long)lf * nn + t, pnl, t0, d, x, y});
      }
    }
  }
  std::stable_sort(hp_pairs.begin(), hp_pairs.end(), [](const HP& a, const HP& b) { return a.node < b.node; });
  std::vector<NearPair> pairs(hp_pairs.size());
  std::vector<long long> node, ptr;
  std::vector<int> panel(hp_pairs.size());
  for (size_t i = 0; i < hp_pairs.size(); ++i) {
    pairs[i] = {hp_pairs[i].x, hp_pairs[i].y, hp_pairs[i].t0, hp_pairs[i].d, hp_pairs[i].panel, 0};
    panel[i] = hp_pairs[i].panel;
    if (i == 0 || hp_pairs[i].node != hp_pairs[i - 1].node) { node.push_back(hp_pairs[i].node); ptr.push_back((long long)i); }
  }
  ptr.push_back((long long)hp_pairs.size());
  if (n_pairs_out) *n_pairs_out = (int64_t)hp_pairs.size();
  if (hp_pairs.empty()) { layer->corrected = true; return VP_OK; }
  vp_tree_s* tr = layer->prog;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevNear d;
  d.n_nodes = (long long)node.size();
  d.n_pairs = (long long)pairs.size();
  NearPair* dp = nullptr;
  int rc;
  if ((rc = dev_upload(tr, pairs, &dp, s))) return rc;
  if ((rc = dev_upload(tr, node, &d.node, s))) return rc;
  if ((rc = dev_upload(tr, ptr, &d.ptr, s))) return rc;
  if ((rc = dev_upload(tr, panel, &d.panel, s))) return rc;
  void* w = nullptr;
  TRY(cudaMalloc(&w, (size_t)d.n_pairs * Q * 4 * sizeof(double)));
  tr->allocs.push_back(w);
  d.dW = static_cast<double*>(w);
  if ((rc = launch_near_weights(tr->T->alpha, g, dp, d.n_pairs, d.dW, s))) return rc;
  const double fl = 2.0 * 16.0 * (double)d.n_pairs * Q;
  const double by = 8.0 * (double)d.n_pairs * Q * 4 + 16.0 * (double)d.n_nodes;
  tr->steps.push_back({7, (int)tr->nears.size(), VP_STAGE_OUTPUT, fl, by});
  tr->flops[VP_STAGE_OUTPUT] += fl;
  tr->bytes[VP_STAGE_OUTPUT] += by;
  tr->nears.push_back(d);
  layer->corrected = true;
  const cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { set_last_cuda(e); return VP_ERR_CUDA; }
  return VP_OK;
}

extern "C" int vp_layer_eval(vp_layer layer, const double* mu, double* u, void* stream) {
  if (!layer || !mu || !u) return VP_ERR_ARG;
  return run_steps(layer->prog, mu, u, u, static_cast<cudaStream_t>(stream));
}

extern "C" int vp_layer_steps(vp_layer layer, const double* mu, double* u, void* stream, int cap, int* n_steps,
                              float* ms, int* info, double* flops, double* bytes) {
  if (!layer) return VP_ERR_ARG;
  return vp_eval_steps(layer->prog, mu, u, u, stream, cap, n_steps, ms, info, flops, bytes);
}

extern "C" void vp_layer_free(vp_layer layer) {
  if (!layer) return;
  vp_tree_free(layer->prog);
  delete layer;
}

// ---------------------------------------------------------------------------
// vp_eval_static: vp_eval without any device allocation.
//
// Some callers cannot call cudaMalloc when they evaluate: code that runs
// under a memory budget fixed before it starts, code that must not touch the
// CUDA allocator while other work holds it, or hosts whose device memory is
// handed out by someone else. For them this variant keeps every work buffer
// of one evaluation (multipole and local coefficients, per-interaction
// contribution slots) in the file-scope array below instead of the tree's own
// buffers. The array is reserved on every GPU that loads the library, until
// the process exits.
#include <mutex>

namespace vp {
namespace {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;  // VP_STATIC_SCRATCH_BYTES in vp.h
constexpr int kMaxDevices = 64;
static __device__ __align__(256) double g_static_scratch[kStaticScratchBytes / sizeof(double)];

std::mutex g_static_mutex;
double* g_static_ptr[kMaxDevices] = {nullptr};

// Device address of the static scratch on the current device (looked up once per device).
int static_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { set_last_cuda(e); return VP_ERR_CUDA; }
  if (dev < 0 || dev >= kMaxDevices) return VP_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) { set_last_cuda(e); return VP_ERR_CUDA; }
    g_static_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_static_ptr[dev];
  return VP_OK;
}

}  // namespace
}  // namespace vp

extern "C" int vp_eval_static(vp_tree tree, const double* f, double* u, double* gradu, void* stream) {
  if (!tree || !f || !u || !gradu) return VP_ERR_ARG;
  const vp_tables_s* T = tree->T;
  if (T->precision != VP_PREC_FP64) return VP_ERR_ARG;
  const size_t nbe = (size_t)tree->n_boxes * T->E;
  const size_t need = 2 * nbe + (size_t)tree->n_lslot * T->C + (size_t)tree->n_uslot * 3 * T->n;
  if (need * sizeof(double) > kStaticScratchBytes) return VP_ERR_ARG;
  double* base = nullptr;
  int rc = static_scratch(&base);
  if (rc != VP_OK) return rc;
  double* mp = base;
  double* loc = mp + nbe;
  double* lslot = loc + nbe;
  double* uslot = lslot + (size_t)tree->n_lslot * T->C;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double* bufs_c[BUF_COUNT] = {f, mp, loc, lslot, uslot};
  double* bufs[BUF_COUNT] = {nullptr, mp, loc, lslot, uslot};
  for (const Step& st : tree->steps) {
    if (st.kind == 2) {
      // the multipole coefficients must start at zero; the other regions are overwritten
      TRY(cudaMemsetAsync(mp, 0, nbe * sizeof(double), s));
    } else if (st.kind == 0) {
      const DevGemm& d = tree->gemms[st.index];
      GemmArgs a = d.args;
      a.A = table_ptr(T, d.table);
      a.X = bufs_c[d.src];
      a.Y = bufs[d.dst];
      if (d.table == T_NEAR) k_gemm_gather_f64<1><<<d.n_tiles, 256, 0, s>>>(a);
      else k_gemm_gather_f64<0><<<d.n_tiles, 256, 0, s>>>(a);
      TRY(cudaGetLastError());
    } else if (st.kind == 1) {
      const DevReduce& d = tree->reduces[st.index];
      ReduceArgs a = d.args;
      a.S = bufs_c[d.src];
      if (a.final_out) { a.u = u; a.g = gradu; } else { a.Y = bufs[d.dst]; }
      const int threads = a.M >= 256 ? 256 : ((a.M + 31) / 32) * 32;
      if (a.M > 4 * threads) return VP_ERR_ARG;  // at most 4 rows per thread (3 p^2 <= 768)
      k_reduce<<<d.n_dst, threads, 0, s>>>(a);
      TRY(cudaGetLastError());
    } else {
      return VP_ERR_ARG;
    }
  }
  return VP_OK;
}
