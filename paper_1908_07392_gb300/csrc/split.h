// Split-precision (sliced operand) contractions: shared declarations.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

struct vp_tables_s;

namespace vp {

constexpr int kSplitSlices = 6;  // 8-bit slices per operand: about 48 significant bits each
constexpr int kSplitKMax = 256;  // K of one contraction (exact fp32 sums need K * 2^16 <= 2^24)

typedef __nv_bfloat16 slice_t;

struct SplitTile {
  int group, m0, col0, ncol;
};

// One sliced operator family, stored tile by tile in the order the GEMM engines stage it: for matrix
// mat, row tile rt (128 rows; rows past M are zero), K step ks (16) and slice s, one 4 KB block
// [2 K chunks of 8][128 rows][8 elements] -- the canonical K-major core-matrix layout (8 rows x 16
// bytes) of the tensor-core operand -- so the S slices of one K step of one row tile are 24 KB of
// contiguous memory that one bulk copy moves. Layout [nmat][nrt][Kpad/16][S][2][128][8] (bf16) and
// row exponents [nmat][M].
struct SplitTable {
  void* A = nullptr;
  int* ea = nullptr;
  int M = 0, K = 0, Kpad = 0, nmat = 0, nrt = 0;
};

// m2m_lo / m2m_hi: the multipole-to-multipole operator split by children (0-1 and 2-3) so that
// every contraction has K = 2C <= 256.
struct SplitTables {
  SplitTable near, s2m, l2t, m2l, m2t, s2l, m2m_lo, m2m_hi, l2l;
};

struct SplitArgs {
  int M, Kpad, out_mode;        // out_mode 0: double-float slot (float2), 1: FP64 overwrite, 2: FP64 accumulate
  int nrt;                      // row tiles of 128 per operator matrix
  int ea_ld;                    // rows per matrix in the row-exponent array (>= M: a launch may use the
                                // leading M rows of its operators)
  const slice_t* A;             // tiled slices (SplitTable)
  const int* ea;
  const slice_t* B;             // sliced vectors [v][S][Kpad]
  const int* eb;
  void* Y;
  const SplitTile* tiles;       // tiles of the engine that runs
  const long long* a_mat;       // per group: matrix index
  const long long* src_vec;     // per column: vector index
  const long long* dst_off;     // per column: destination offset (elements of 8 bytes)
};

struct DFReduceArgs {
  int M, n, final_out;
  long long N;
  const long long* dst_off;
  const long long* ptr;
  const long long* slot;
  const void* S;
  double* Y;
  double* u;
  double* g;
};

// GEMM engines for the sliced contraction: warp-level mma.sync on 128 x 64 tiles, tcgen05 with tensor
// memory on 128 x 128 tiles, mma.sync on 64 x 32 tiles (four times the CTAs of the first: for the
// small, latency-bound launches of the coarse levels), and tcgen05 on 128 x 64 tiles with two
// accumulator sets in tensor memory (the epilogue of a tile overlaps the MMAs of the next: for
// contractions with short K, whose tiles are bound by the epilogue), and tcgen05 on transposed 128 x
// 128 tiles (columns as the MMA's 128 rows, operator rows as its N: for operators of at most 128
// rows, whose own rows would leave tensor-memory lanes idle). vp_autotune chooses per launch shape.
constexpr int kEngineMmaSync = 0, kEngineTcgen05 = 1, kEngineMmaSmall = 2, kEngineTcgen05N64 = 3,
              kEngineTcgen05T = 4;
constexpr int kEngines = 5;
constexpr int kSplitBM = 128;                                  // rows of a table tile (the tiled layout's unit)
constexpr int kSplitBMe[kEngines] = {128, 128, 64, 128, 128};  // rows per GEMM tile, by engine
constexpr int kSplitBN[kEngines] = {64, 128, 32, 64, 128};     // columns per GEMM tile, by engine

int build_split(vp_tables_s* T, cudaStream_t s);
void free_split_tables(vp_tables_s* T);
int prepare_split_launch();
// short_ctas: tcgen05 CTAs take two tiles each (so other kernels can interleave) instead of one
// persistent CTA per SM.
int launch_split_gemm(const SplitArgs& a, int n_tiles, cudaStream_t s, int engine, int short_ctas = 0);
// Read and clear the flag that a bounded wait of the tcgen05 engine gave up.
int read_split_error(int* flag);
// Run a kernel whose bounded wait on an mbarrier nothing arrives at gives up after `budget` clocks.
int selftest_wait(long long budget, cudaStream_t s);
int launch_slice_list(const double* X, const long long* base, const long long* vid, long long nlist, int K, int kseg,
                      long long seg_stride, long long cstride, void* out, int* eb, cudaStream_t s);
int launch_reduce_df(const DFReduceArgs& a, int n_dst, cudaStream_t s);
int split_kpad(int K);

}  // namespace vp
