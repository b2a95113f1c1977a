// Split-precision contractions on the tensor cores (VP_PREC_SPLIT).
//
// An FP64 product y = A x (A an operator table, x a coefficient or nodal
// vector) is computed from exact integer slices, in the manner of Ozaki's
// error-free splitting of matrix products (Ozaki, Ogita, Oishi and Rump,
// Numer. Algorithms 59, 2012):
//   * each row r of A is scaled by 2^-ea[r] (ea[r] = exponent of the row's
//     largest entry, so the scaled row lies in (-1, 1)) and written in S = 6
//     balanced base-256 digits: A[r,k] = 2^ea[r] sum_i a_i[r,k] 2^(-8(i+1))
//     up to 2^(ea[r] - 49); each vector x likewise with one exponent eb;
//   * slice i holds a_i 2^(-8(i+1)) in bf16: every digit (|a_0| <= 256,
//     |a_i| <= 128 for i >= 1) is exactly representable and the power-of-two
//     scale keeps it exact, so every product of two slices is exact;
//   * products with the same weight w = i + j are integer multiples of one
//     power of two; their sum over K <= 256 stays below 2^24 of that unit for
//     w <= 1 (and within 2^-24 of it at w = 2), so an fp32 accumulator per
//     weight w = 0, 1, 2 holds it exactly; weights w >= 3 share a fourth
//     accumulator whose rounding is below 2^-48 of the result;
//   * the four sums are added in double-float (two fp32) and scaled by
//     2^(ea[r] + eb) exactly. Products with i + j > S - 1 are dropped.
// Two engines run the same arithmetic: warp-level mma.sync (m16n8k16 bf16),
// and tcgen05.mma with the accumulators in tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <new>
#include <vector>

#include "plan.h"
#include "split.h"
#include "vp_internal.h"

namespace vp {

namespace {

#define TRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_last_cuda(e_); return e_ == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA; } } while (0)

constexpr int kAcc = 4;  // accumulators: weights 0, 1, 2 and the tail

// Balanced base-256 digits of |x| * 2^(8S - e) (|x| < 2^e), taken straight from the FP64 bit pattern
// with integer arithmetic: T = round(|x| 2^(8S-e)) < 2^(8S) (+1 from rounding), then the digits from the
// least significant up, each moved into [-128, 127] with a carry, the leading one in [0, 256]; the sign
// of x is applied to every digit. Slice i receives digit_i * 2^(-8(i+1)) (exact in bf16).
template <int S>
__device__ inline void digits(double x, int e, slice_t* out, size_t stride) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  int ex = (int)((bits >> 52) & 0x7ff);
  unsigned long long m = bits & ((1ull << 52) - 1);
  if (ex) m |= 1ull << 52;
  else ex = 1;
  const int sh = ex - 1075 + 8 * S - e;
  unsigned long long T;
  if (m == 0 || sh <= -64) T = 0;
  else if (sh >= 0) T = m << sh;
  else T = (m + (1ull << (-sh - 1))) >> (-sh);
  int dig[S];
#pragma unroll
  for (int i = S - 1; i >= 1; --i) {
    int r = (int)(T & 255ull);
    T >>= 8;
    if (r >= 128) { r -= 256; T += 1; }
    dig[i] = r;
  }
  dig[0] = (int)T;
  const bool neg = (bits >> 63) != 0;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    const float v = (float)(neg ? -dig[i] : dig[i]) * __int_as_float((127 - 8 * (i + 1)) << 23);
    out[i * stride] = __float2bfloat16_rn(v);
  }
}

// Exponent e with |v| < 2^e for v = max |x| > 0 (0 for v = 0).
__device__ inline int exponent_of(double v) {
  int e = 0;
  if (v > 0.0) frexp(v, &e);
  return e;
}

// Slice rows of a batch of matrices: A[mat][r][k] (row stride lda, matrix stride mstride) -> the
// tiled layout of SplitTable (out[mat][r / 128][k / 16][s][(k % 16) / 8][r % 128][k % 8]; the caller
// zeroes the padding rows) and ea[mat][r]. One warp per row.
template <int S>
__global__ void k_slice_rows(const double* __restrict__ A, long long mstride, int lda, int M, int K, int Kpad,
                             int nmat, int nrt, slice_t* __restrict__ out, int* __restrict__ ea) {
  const long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= (long long)nmat * M) return;
  const long long mat = row / M;
  const int r = (int)(row - mat * M);
  const double* a = A + mat * mstride + (long long)r * lda;
  double mx = 0.0;
  for (int k = lane; k < K; k += 32) mx = fmax(mx, fabs(a[k]));
  for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int e = exponent_of(mx);
  const int nks = Kpad / 16;
  slice_t* o = out + (mat * nrt + (r >> 7)) * (long long)nks * S * 2048 + (r & 127) * 8;
  for (int k = lane; k < Kpad; k += 32)
    digits<S>(k < K ? a[k] : 0.0, e, o + (long long)(k >> 4) * S * 2048 + ((k >> 3) & 1) * 1024 + (k & 7), 2048);
  if (lane == 0) ea[mat * M + r] = e;
}

// Slice a list of vectors. Vector v (v < nlist) has identifier id = vid ? vid[v] : v and elements
// x_k = X[b + (k / kseg) * seg_stride + k % kseg], k < K, b = base ? base[v] : v * cstride;
// output out[id][Kpad / 16][s][16] (the S slices of each K step of 16 are contiguous, so one
// column of a K step is one 32 S-byte block for the GEMM engines' gathers) and eb[id]. One warp
// per vector.
template <int S>
__global__ void k_slice_list(const double* __restrict__ X, const long long* __restrict__ base,
                             const long long* __restrict__ vid, long long nlist, int K, int kseg,
                             long long seg_stride, long long cstride, int Kpad, slice_t* __restrict__ out,
                             int* __restrict__ eb) {
  const long long v = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (v >= nlist) return;
  const long long b = base ? base[v] : v * cstride;
  const long long id = vid ? vid[v] : v;
  double mx = 0.0;
  for (int k = lane; k < K; k += 32) {
    const int sg = k / kseg;
    mx = fmax(mx, fabs(X[b + sg * seg_stride + (k - sg * kseg)]));
  }
  for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int e = exponent_of(mx);
  slice_t* o = out + id * (long long)S * Kpad;
  for (int k = lane; k < Kpad; k += 32) {
    const int sg = k / kseg;
    digits<S>(k < K ? X[b + sg * seg_stride + (k - sg * kseg)] : 0.0, e, o + (k >> 4) * (S * 16) + (k & 15), 16);
  }
  if (lane == 0) eb[id] = e;
}

__device__ inline void df_add(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  const float l = __fadd_rn(lo, err);
  const float t = __fadd_rn(s, l);
  lo = __fsub_rn(l, __fsub_rn(t, s));
  hi = t;
}

// s + e = a + b exactly (Knuth's TwoSum, no ordering of |a|, |b| assumed).
__device__ inline void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// The four weight-group sums of one output as a double-float (h, l): groups 0, 1 and 2 enter through
// TwoSums (exact), so only the two rounding errors those leave (each below 2^-24 of a partial sum)
// and group 3 (the tail, below 2^-24 of the scale) are added in fp32; a last TwoSum renormalises.
// h + l is within 2^-23 (|e| + |e2| + |a3|) <= about 2^-47 of the partial sums of the exact total.
// (Group 2 added in fp32 as well costs 2^-24 of it, which cancellation in the contraction makes
// visible: gradients of the star workload at 2e-9 instead of 1e-10.)
__device__ inline void fold4(float a0, float a1, float a2, float a3, float& h, float& l) {
  float s, e, s2, e2;
  two_sum(a0, a1, s, e);
  two_sum(s, a2, s2, e2);
  two_sum(s2, __fadd_rn(__fadd_rn(e, e2), a3), h, l);
}

// 2^e as a float / double (e in the normal range of the type).
__device__ inline float pow2f(int e) { return __int_as_float((e + 127) << 23); }
__device__ inline double pow2d(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

// One output element: double-float (h, l) times 2^e, as a double-float slot (out_mode 0) or in
// FP64 (out_mode 1 overwrites, 2 adds to `old`, the value the destination held before the launch).
// Scaling by a power of two is exact (ldexp only where 2^e itself is not a normal number). Callers
// with out_mode 2 read the old values of a group of outputs first, so that the reads of the group
// are in flight together instead of one read-add-store chain per element.
// The 8 bytes store_out would write for out_mode 0 (double-float slot) or 1 (FP64), as a double.
__device__ inline double out_value(const SplitArgs& a, float h, float l, int e) {
  if (a.out_mode == 0) {
    float2 o;
    if (e >= -126 && e <= 127) {
      const float sc = pow2f(e);
      o.x = h * sc;
      o.y = l * sc;
    } else {
      o.x = ldexpf(h, e);
      o.y = ldexpf(l, e);
    }
    return __hiloint2double(__float_as_int(o.y), __float_as_int(o.x));
  }
  const double hl = (double)h + (double)l;
  return (e >= -1022 && e <= 1023) ? hl * pow2d(e) : ldexp(hl, e);
}

__device__ inline void store_out(const SplitArgs& a, long long dst, int row, float h, float l, int e, double old) {
  if (a.out_mode == 0) {
    float2 o;
    if (e >= -126 && e <= 127) {
      const float sc = pow2f(e);
      o.x = h * sc;
      o.y = l * sc;
    } else {
      o.x = ldexpf(h, e);
      o.y = ldexpf(l, e);
    }
    reinterpret_cast<float2*>(a.Y)[dst + row] = o;
  } else {
    const double hl = (double)h + (double)l;
    const double val = (e >= -1022 && e <= 1023) ? hl * pow2d(e) : ldexp(hl, e);
    reinterpret_cast<double*>(a.Y)[dst + row] = (a.out_mode == 2) ? old + val : val;
  }
}

__device__ inline void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(n));
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
template <int N>
__device__ inline void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// ------------------------------------------------------------------ engine 0: mma.sync

constexpr int kMKC = 32, kMPitch = kMKC + 8;             // K chunk and shared row pitch (elements)

__device__ inline void ldmatrix_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}

__device__ inline void mma16816(float* c, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Tile BM x BN, warps of 32 x 32 (BM/32 along M, BN/32 along N), K in chunks of 32, double buffered.
template <int S, int BM, int BN>
__global__ void __launch_bounds__(BM * BN / 32) k_split_gemm(SplitArgs a) {
  constexpr int NT = BM * BN / 32, WM = BM / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  slice_t* As = reinterpret_cast<slice_t*>(smem_raw);                  // [2][S][BM][pitch]
  slice_t* Bs = As + 2 * S * BM * kMPitch;                              // [2][S][BN][pitch]
  const SplitTile tile = a.tiles[blockIdx.x];
  const long long mat = a.a_mat[tile.group];
  // this tile's rows in the tiled operator layout: [K step][slice][chunk][128 rows][8], rows from
  // m0 % 128 within the table tile
  const slice_t* Ag = a.A + (mat * a.nrt + (tile.m0 >> 7)) * (long long)(a.Kpad / 16) * S * 2048 + (tile.m0 & 127) * 8;
  const int* ea = a.ea + mat * a.ea_ld;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp % WM, wn = warp / WM;  // WM warps along M (32 rows), BN/32 along N (32 columns)
  const int gid = lane >> 2, tig = lane & 3;

  auto load_chunk = [&](int buf, int k0) {
    for (int e = tid; e < S * BM * 4; e += NT) {
      const int sl = e / (BM * 4), rem = e % (BM * 4);
      const int c = rem / BM, r = rem % BM;  // K chunk of 8 (0..3 within the 32), row
      const slice_t* src = Ag + ((long long)(((k0 >> 4) + (c >> 1)) * S + sl) * 2 + (c & 1)) * 1024 + r * 8;
      cp_async16(As + ((buf * S + sl) * BM + r) * kMPitch + c * 8, src, true);  // padding rows are zeros
    }
    // one column's two K steps of 16 are 4 S contiguous 16-byte chunks (step, slice, half)
    for (int e = tid; e < S * BN * 4; e += NT) {
      const int col = e / (S * 4), w = e % (S * 4);
      const int ks = w / (S * 2), sl = (w >> 1) % S, h = w & 1;
      const bool ok = col < tile.ncol;
      const long long v = ok ? a.src_vec[tile.col0 + col] : 0;
      const slice_t* src = a.B + v * S * (long long)a.Kpad + (k0 >> 4) * (S * 16) + w * 8;
      cp_async16(Bs + ((buf * S + sl) * BN + col) * kMPitch + ks * 16 + h * 8, src, ok);
    }
    cp_async_commit();
  };

  float acc[kAcc][2][4][4];
#pragma unroll
  for (int w = 0; w < kAcc; ++w)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[w][i][j][c] = 0.f;

  const int nchunks = a.Kpad / kMKC;
  load_chunk(0, 0);
  for (int ch = 0; ch < nchunks; ++ch) {
    const int buf = ch & 1;
    if (ch + 1 < nchunks) {
      load_chunk(buf ^ 1, (ch + 1) * kMKC);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kMKC / 16; ++ks) {
      unsigned bf[S][4][2];
#pragma unroll
      for (int j = 0; j < S; ++j) {
        const slice_t* Bb = Bs + ((buf * S + j) * BN + wn * 32) * kMPitch;
#pragma unroll
        for (int nt2 = 0; nt2 < 2; ++nt2) {
          unsigned r0, r1, r2, r3;
          ldmatrix_x4(r0, r1, r2, r3,
                      Bb + (nt2 * 16 + (lane & 7) + ((lane >> 4) << 3)) * kMPitch + ks * 16 + ((lane >> 3) & 1) * 8);
          bf[j][nt2 * 2][0] = r0; bf[j][nt2 * 2][1] = r1;
          bf[j][nt2 * 2 + 1][0] = r2; bf[j][nt2 * 2 + 1][1] = r3;
        }
      }
#pragma unroll
      for (int i = 0; i < S; ++i) {
        const slice_t* Ab = As + ((buf * S + i) * BM + wm * 32) * kMPitch;
        unsigned af[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
          ldmatrix_x4(af[mt][0], af[mt][1], af[mt][2], af[mt][3],
                      Ab + (mt * 16 + (lane & 15)) * kMPitch + ks * 16 + (lane >> 4) * 8);
#pragma unroll
        for (int j = 0; i + j < S; ++j) {
          const int w = (i + j < kAcc - 1) ? i + j : kAcc - 1;
#pragma unroll
          for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) mma16816(acc[w][mt][nt], af[mt], bf[j][nt]);
        }
      }
    }
    __syncthreads();
  }

#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    bool cok[2];
    int eb[2];
    long long dst[2];
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
      const int col = wn * 32 + nt * 8 + tig * 2 + cc;
      cok[cc] = col < tile.ncol;
      eb[cc] = cok[cc] ? a.eb[a.src_vec[tile.col0 + col]] : 0;
      dst[cc] = cok[cc] ? a.dst_off[tile.col0 + col] : 0;
    }
    double old[2][2][2] = {};
    if (a.out_mode == 2) {
#pragma unroll
      for (int cc = 0; cc < 2; ++cc)
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int rr = 0; rr < 2; ++rr) {
            const int row = tile.m0 + wm * 32 + mt * 16 + gid + rr * 8;
            if (cok[cc] && row < a.M) old[cc][mt][rr] = reinterpret_cast<const double*>(a.Y)[dst[cc] + row];
          }
    }
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
      if (!cok[cc]) continue;
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
          const int row = tile.m0 + wm * 32 + mt * 16 + gid + rr * 8;
          if (row >= a.M) continue;
          float h, l;
          fold4(acc[0][mt][nt][rr * 2 + cc], acc[1][mt][nt][rr * 2 + cc], acc[2][mt][nt][rr * 2 + cc],
                acc[3][mt][nt][rr * 2 + cc], h, l);
          store_out(a, dst[cc], row, h, l, ea[row] + eb[cc], old[cc][mt][rr]);
        }
    }
  }
}

size_t mma_smem_bytes(int S, int BM, int BN) { return (size_t)2 * S * (BM + BN) * kMPitch * sizeof(slice_t); }

// ------------------------------------------------------------------ engine 1: tcgen05
//
// Persistent and warp-specialised: one CTA per SM walks the tile list (tile t, t + gridDim.x, ...).
//  * warps 0-3 (producers) stage the operands of every K step of 16 into a 4-stage ring in the
//    canonical K-major layout without swizzle (8-row x 16-byte core matrices): the operator slices
//    (A), stored in that layout tile by tile, by one bulk copy (cp.async.bulk, 24 KB) issued by
//    thread 0, whose bytes complete on the stage's `fullA` mbarrier (next core matrix along K 2048
//    bytes further, next 8-row group 128 bytes further); the gathered source columns (B) by
//    cp.async (next core matrix along K 128 bytes, next 8-column group 256 bytes further), each
//    thread's copies arriving on the stage's `full` mbarrier when they land
//    (cp.async.mbarrier.arrive); a producer waits only for free stages. The ring runs on across
//    tiles, so the next tile's operands stream in while the current one is drained. (Moving A by a
//    tensor map whose boxes are 16 bytes wide -- the same layout built by the TMA unit -- made the
//    whole K step 1.7x slower: narrow boxes cost the unit far more than one contiguous copy.)
//  * warps 4 .. 15 (epilogue) read the accumulators (warp w: tensor-memory lanes 32 (w % 4) .. + 31,
//    one accumulator row per thread, every third block of 16 columns), fold them in double-float and
//    store. (Three warps per lane quadrant: the epilogue is the part of a tile that the MMAs wait
//    for, and four producer warps issue a K step's copies easily.)
//  * warp 16 (one thread) waits on `full`, fences the generic-proxy writes of the stage against the
//    async proxy, issues tcgen05.mma (kind::f16, bf16 operands, M = 128, N = BN, K = 16) into four
//    fp32 accumulators in tensor memory (one per weight group) and commits to the stage's `empty`
//    mbarrier; after a tile's last step it commits to `acc`, and it starts the next tile once the
//    epilogue has arrived on `tmem_free`.
// Every wait is bounded and also ends once another thread has given up; decisions taken by the
// epilogue group are made uniform with a barrier reduction. A kernel that gave up raises a flag,
// lets its issued MMAs finish (bounded), skips its remaining stores and releases tensor memory.

__device__ int g_split_error = 0;

constexpr int kTcProducers = 128;                 // warps 0-3
#ifndef VP_TC_EPILOGUE_WARPS
#define VP_TC_EPILOGUE_WARPS 12
#endif
constexpr int kTcEpilogue = 32 * VP_TC_EPILOGUE_WARPS;  // warps 8 .. 8 + warps - 1
constexpr int kTcEpiParts = VP_TC_EPILOGUE_WARPS / 4;   // epilogue warps per tensor-memory lane quadrant
constexpr int kTcMmaWarp = (kTcProducers + kTcEpilogue) / 32;
constexpr int kTcThreads = kTcProducers + kTcEpilogue + 32;
constexpr int kTcKC = 16;                         // K per stage
constexpr int kTcStages = 4;
constexpr int kTcCols = 512;                      // tensor-memory columns allocated per CTA
constexpr int kTcA = kSplitBM * kTcKC;            // elements per A slice tile
static_assert(kSplitBN[kEngineTcgen05] == 128 && kSplitBN[kEngineTcgen05N64] == 64, "tcgen05 tile widths");
static_assert(kSplitBM == 128 && kTcProducers % 128 == 0 && kTcEpiParts * 128 == kTcEpilogue, "thread mapping");

// Tile width BN (columns) of a tcgen05 engine: the four accumulators take 4 BN tensor-memory
// columns, so at BN = 64 two sets fit and the MMAs of a tile run while the epilogue drains the
// previous one (at BN = 128 the epilogue and the next tile's MMAs alternate).
template <int BN>
struct TcShape {
  static constexpr int kB = BN * kTcKC;           // elements per B slice tile
  static constexpr int kAccCols = kAcc * BN;      // tensor-memory columns of one accumulator set
  static constexpr int kBufs = kTcCols / kAccCols;
  static_assert(kBufs >= 1 && kBufs * kAccCols == kTcCols, "accumulator sets fill tensor memory");
};

__device__ inline unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ inline unsigned long long umma_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((saddr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);  // version 1, no swizzle
}

__device__ inline void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ inline void mbar_arrive(unsigned long long* bar) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar)) : "memory");
}

// One tcgen05.mma kind::f16 (A and B from shared-memory descriptors) with an A-collector usage:
// U = 0 none, 1 fill, 2 use, 3 lastuse.
template <int U>
__device__ inline void umma_f16(unsigned d_tmem, unsigned long long da, unsigned long long db, unsigned idesc,
                                unsigned accum) {
  if constexpr (U == 0) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
                 "l"(da), "l"(db), "r"(idesc), "r"(accum));
  } else if constexpr (U == 1) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
                 "l"(da), "l"(db), "r"(idesc), "r"(accum));
  } else if constexpr (U == 2) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16.collector::a::use [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
                 "l"(da), "l"(db), "r"(idesc), "r"(accum));
  } else {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n}\n" ::"r"(
                     d_tmem),
                 "l"(da), "l"(db), "r"(idesc), "r"(accum));
  }
}

// The S(S+1)/2 slice products of one K step, fully unrolled: product (i, j) accumulates into the
// weight group w = min(i + j, 3); A slice i is read into the A collector once and reused by its
// S - i products. FIRST: step 0 of a tile, where the first product of each group overwrites it.
// W: columns of one accumulator; KA, KB: strides between the slice tiles of the A and B operands in
// shared memory (16-byte units).
template <int S, int W, int KA, int KB, bool FIRST>
__device__ __forceinline__ void mma_kstep(unsigned tmem, unsigned long long da, unsigned long long db, unsigned idesc) {
#pragma unroll
  for (int i = 0; i < S; ++i) {
#pragma unroll
    for (int j = 0; i + j < S; ++j) {
      constexpr int kA = KA, kB = KB;
      const int w = (i + j < kAcc - 1) ? i + j : kAcc - 1;
      const unsigned d_tmem = tmem + (unsigned)(w * W);
      const unsigned long long a = da + (unsigned long long)(i * kA), b = db + (unsigned long long)(j * kB);
      const unsigned accum = (FIRST && i == 0 && j == w) ? 0u : 1u;
      const int uses = S - i;
      if (uses == 1) umma_f16<0>(d_tmem, a, b, idesc, accum);
      else if (j == 0) umma_f16<1>(d_tmem, a, b, idesc, accum);
      else if (j < uses - 1) umma_f16<2>(d_tmem, a, b, idesc, accum);
      else umma_f16<3>(d_tmem, a, b, idesc, accum);
    }
  }
}

__device__ inline void umma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}

// Bounded wait for the completion of phase `parity` of an mbarrier: false if it gave up (~2 s) or
// if *abort became nonzero meanwhile.
__device__ inline bool mbar_wait(unsigned long long* bar, unsigned parity, volatile int* abort = nullptr,
                                 long long budget = 4000000000ll) {
  const unsigned a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    unsigned done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (abort && *abort) return false;
    if (clock64() - t0 > budget) return false;
  }
}

// Exercises the give-up path of the bounded waits: one thread waits on an mbarrier that nothing
// arrives at, with a budget of `budget` clocks, and raises the same device flag as the GEMM kernel.
__global__ void k_wait_selftest(long long budget) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;\n");
  if (!mbar_wait(&bar, 0, nullptr, budget)) atomicExch(&g_split_error, 1);
}

// Named barrier 1 over the epilogue warps, returning the AND of `pred` over them (uniform).
__device__ inline bool epi_all(bool pred) {
  unsigned r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.and.pred q, 1, %2, p;\nselp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((unsigned)pred), "n"(kTcEpilogue)
      : "memory");
  return r != 0;
}

// TR = 0: D [operator rows x columns] = operator slices (A) x gathered vectors (B), N = BN.
// TR > 0 (operators of at most TR <= 128 rows, BN = 128): the transposed product D^T [columns x rows]
// = gathered vectors (A, M = 128) x operator slices (B, N = TR), so every tensor-memory lane -- and
// every epilogue thread -- holds one of the tile's 128 columns even when the operator has only 81
// rows (the multipole and local operators). The shared-memory layouts are the same; only the
// descriptors trade places.
template <int S, int BN, int TR>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_split_gemm_tc(SplitArgs a, int n_tiles) {
  static_assert(TR == 0 || (BN == 128 && TR % 16 == 0 && TR <= 128), "transposed tiles");
  constexpr int kTcB = TcShape<BN>::kB;
  constexpr int kAccCols = TR ? kAcc * TR : TcShape<BN>::kAccCols, kBufs = TR ? 1 : TcShape<BN>::kBufs;
  constexpr int kQ = BN * 2 * S / kTcProducers;  // 16-byte B chunks per producer thread and K step
  static_assert(kQ * kTcProducers == BN * 2 * S, "B chunks divide among the producers");
  extern __shared__ __align__(128) unsigned char smem_tc[];
  slice_t* As = reinterpret_cast<slice_t*>(smem_tc);  // [stages][S][kTcA]
  slice_t* Bs = As + kTcStages * S * kTcA;              // [stages][S][kTcB]
  __shared__ __align__(8) unsigned long long full[kTcStages], fullA[kTcStages], empty[kTcStages], accbar[kBufs],
      tmem_free[kBufs], donebar;
  __shared__ unsigned tmem_base_sh;
  __shared__ volatile int abort_sh;
  __shared__ long long col_dst[BN];  // current tile, per column: destination offset, source exponent
  __shared__ int col_e[BN];
  // transposed tiles: per epilogue warp, eight outputs of its 32 lanes' destinations on their way to
  // coalesced stores
  __shared__ __align__(16) double stage[TR ? kTcEpilogue / 32 : 1][32][8];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == kTcMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base_sh)),
                 "n"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&full[s], kTcProducers);  // cp.async copies of the B operand
      mbar_init(&fullA[s], 1);            // bulk copy of the A operand (byte count)
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < kBufs; ++b) {
      mbar_init(&accbar[b], 1);
      mbar_init(&tmem_free[b], kTcEpilogue);
    }
    mbar_init(&donebar, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const unsigned tmem = tmem_base_sh;
  const int nk = a.Kpad / kTcKC;

  if (warp < kTcProducers / 32) {
    // ---- producers: a K step of the gathered operand is BN columns x 2 S chunks of 16 bytes; a
    // column's chunks (slice, half) are contiguous in global memory, so consecutive threads take
    // consecutive chunks: thread t copies chunks q = t + 128 i, i < kQ (column q / 2S, slice
    // (q % 2S) / 2, half q % 2)
    const slice_t* bsrc[kQ];
    int bdst[kQ];
    bool bok[kQ];
    long long g = 0;  // ring step across tiles
    bool ok = true;
    for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
      const SplitTile tile = a.tiles[t];
      // A: the S slices of K step k of this row tile are one contiguous block of S x 4 KB
      const slice_t* ablk = a.A + (a.a_mat[tile.group] * a.nrt + (tile.m0 >> 7)) * (long long)nk * S * kTcA;
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        const int q = tid + kTcProducers * i;
        const int col = q / (2 * S), w = q % (2 * S);
        const int sl = w >> 1, c = w & 1;
        bok[i] = col < tile.ncol;
        const long long v = bok[i] ? a.src_vec[tile.col0 + col] : 0;
        bsrc[i] = a.B + v * S * (long long)a.Kpad + w * 8;
        bdst[i] = sl * kTcB + ((col >> 3) * 2 + c) * 64 + (col & 7) * 8;
      }
      for (int k = 0; k < nk; ++k, ++g) {
        const int st = (int)(g % kTcStages);
        if (g >= kTcStages && !mbar_wait(&empty[st], (unsigned)((g / kTcStages) - 1) & 1u, &abort_sh)) {
          ok = false;
          break;
        }
        if (tid == 0) {
          // A operand: one bulk copy of the stage's S slice tiles, completion counted in bytes
          asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
                           smem_u32(&fullA[st])),
                       "n"(S * kTcA * (int)sizeof(slice_t))
                       : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                  smem_u32(As + st * S * kTcA)),
              "l"(ablk + (long long)k * S * kTcA), "n"(S * kTcA * (int)sizeof(slice_t)), "r"(smem_u32(&fullA[st]))
              : "memory");
        }
#pragma unroll
        for (int i = 0; i < kQ; ++i) cp_async16(Bs + st * S * kTcB + bdst[i], bsrc[i] + k * (S * 16), bok[i]);
        // arrives on full[st] once this thread's copies so far have landed; the thread moves on
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(&full[st])) : "memory");
      }
    }
    cp_async_wait_all();
    if (!ok) abort_sh = 1;
    if (tid == 0) {
      // no bulk copy may still be in flight when the CTA ends (after giving up too): wait for the
      // copies of the last stages issued (earlier ones were consumed by the MMA warp)
      for (long long q = (g > kTcStages ? g - kTcStages : 0); q < g; ++q)
        mbar_wait(&fullA[q % kTcStages], (unsigned)(q / kTcStages) & 1u);
    }
  } else if (warp < kTcMmaWarp) {
    // ---- epilogue
    if constexpr (TR > 0) {
      // transposed tiles: lane = column of the tile (vector, destination), tensor-memory column =
      // operator row
      const int e = tid - kTcProducers;
      const int q = warp & 3, part = (warp - kTcProducers / 32) >> 2;
      int it = 0;
      for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++it) {
        const SplitTile tile = a.tiles[t];
        for (int o = e; o < TR; o += kTcEpilogue) col_e[o] = o < a.M ? a.ea[a.a_mat[tile.group] * a.ea_ld + o] : 0;
        const int pc = q * 32 + lane;
        const bool pok = pc < tile.ncol;
        const long long dst = pok ? a.dst_off[tile.col0 + pc] : 0;
        const int ebv = pok ? a.eb[a.src_vec[tile.col0 + pc]] : 0;
        const bool acc_ok = mbar_wait(&accbar[0], (unsigned)it & 1u, &abort_sh);
        // uniform over the epilogue group (also publishes the row exponents written above)
        if (!epi_all(acc_ok && !abort_sh)) {
          abort_sh = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n");
#pragma unroll 1
        for (int cb = part; cb < TR / 16; cb += kTcEpiParts) {
          if (cb * 16 >= a.M) break;
          float vv[kAcc][16];
#pragma unroll
          for (int w = 0; w < kAcc; ++w) {
            const unsigned taddr = tmem + ((unsigned)(q * 32) << 16) + (unsigned)(w * TR + cb * 16);
            unsigned rr[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];\n"
                : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]),
                  "=r"(rr[7]), "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]),
                  "=r"(rr[14]), "=r"(rr[15])
                : "r"(taddr));
#pragma unroll
            for (int cc = 0; cc < 16; ++cc) vv[w][cc] = __uint_as_float(rr[cc]);
          }
          asm volatile("tcgen05.wait::ld.sync.aligned;\n");
          if (a.out_mode != 2 && cb * 16 + 16 <= a.M) {
            // a full block of 16 outputs: each lane forms its 8-byte values (double-float slot or
            // FP64), eight at a time, into the warp's staging rows; then lanes 8 g .. 8 g + 7 store
            // eight consecutive outputs of destination 4 i + g, four destinations per instruction
            double (*stg)[8] = stage[(warp - kTcProducers / 32)];
#pragma unroll
            for (int c8 = 0; c8 < 16; c8 += 8) {
#pragma unroll
              for (int cc = 0; cc < 8; ++cc) {
                const int o = cb * 16 + c8 + cc;
                float h, l;
                fold4(vv[0][c8 + cc], vv[1][c8 + cc], vv[2][c8 + cc], vv[3][c8 + cc], h, l);
                stg[lane][cc] = out_value(a, h, l, col_e[o] + ebv);
              }
              __syncwarp();
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const int src = 4 * i + (lane >> 3);
                const long long d = __shfl_sync(0xffffffffu, dst, src);
                if (q * 32 + src < tile.ncol)
                  reinterpret_cast<double*>(a.Y)[d + cb * 16 + c8 + (lane & 7)] = stg[src][lane & 7];
              }
              __syncwarp();
            }
          } else if (pok && a.out_mode != 2) {
#pragma unroll
            for (int cc = 0; cc < 16; ++cc) {
              const int o = cb * 16 + cc;
              if (o >= a.M) break;
              float h, l;
              fold4(vv[0][cc], vv[1][cc], vv[2][cc], vv[3][cc], h, l);
              store_out(a, dst, o, h, l, col_e[o] + ebv, 0.0);
            }
          } else if (pok) {
            // accumulating launch: fold, read the old values of eight outputs together, store
#pragma unroll
            for (int cc = 0; cc < 16; ++cc) {
              float h, l;
              fold4(vv[0][cc], vv[1][cc], vv[2][cc], vv[3][cc], h, l);
              vv[0][cc] = h;
              vv[1][cc] = l;
            }
#pragma unroll
            for (int c8 = 0; c8 < 16; c8 += 8) {
              double old[8];
#pragma unroll
              for (int cc = 0; cc < 8; ++cc) {
                const int o = cb * 16 + c8 + cc;
                old[cc] = o < a.M ? reinterpret_cast<const double*>(a.Y)[dst + o] : 0.0;
              }
#pragma unroll
              for (int cc = 0; cc < 8; ++cc) {
                const int o = cb * 16 + c8 + cc;
                if (o < a.M) store_out(a, dst, o, vv[0][c8 + cc], vv[1][c8 + cc], col_e[o] + ebv, old[cc]);
              }
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n");
        mbar_arrive(&tmem_free[0]);
        asm volatile("bar.sync 1, %0;\n" ::"n"(kTcEpilogue) : "memory");
      }
    } else {

    const int e = tid - kTcProducers;
    // warp w reads tensor-memory lanes 32 (w % 4) .. + 31; the kTcEpiParts warps of a quadrant share
    // its column blocks
    const int q = warp & 3, part = (warp - kTcProducers / 32) >> 2;
    int it = 0;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++it) {
      const SplitTile tile = a.tiles[t];
      const int buf = it % kBufs;
      if (e % (kTcEpilogue / BN) == 0) {
        const int col = e / (kTcEpilogue / BN);
        const bool cok = col < tile.ncol;
        const long long v = cok ? a.src_vec[tile.col0 + col] : 0;
        col_dst[col] = cok ? a.dst_off[tile.col0 + col] : 0;
        col_e[col] = cok ? a.eb[v] : 0;
      }
      const int row = tile.m0 + q * 32 + lane;
      const bool row_ok = row < a.M;
      const int era = row_ok ? a.ea[a.a_mat[tile.group] * a.ea_ld + row] : 0;
      const bool acc_ok = mbar_wait(&accbar[buf], (unsigned)(it / kBufs) & 1u, &abort_sh);
      // uniform over the epilogue group (also publishes the column metadata written above)
      if (!epi_all(acc_ok && !abort_sh)) {
        abort_sh = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n");
#pragma unroll 1
      for (int cb = part; cb < BN / 16; cb += kTcEpiParts) {
        if (cb * 16 >= tile.ncol) break;
        float vv[kAcc][16];
#pragma unroll
        for (int w = 0; w < kAcc; ++w) {
          const unsigned taddr =
              tmem + ((unsigned)(q * 32) << 16) + (unsigned)(buf * kAccCols + w * BN + cb * 16);
          unsigned rr[16];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
              "[%16];\n"
              : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]),
                "=r"(rr[7]), "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]),
                "=r"(rr[14]), "=r"(rr[15])
              : "r"(taddr));
#pragma unroll
          for (int cc = 0; cc < 16; ++cc) vv[w][cc] = __uint_as_float(rr[cc]);
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;\n");
        if (row_ok && a.out_mode != 2 && cb * 16 + 16 <= tile.ncol) {
          // a full block of 16 columns: no per-column exit, so the columns' independent chains
          // (metadata load, fold, store) interleave
#pragma unroll
          for (int cc = 0; cc < 16; ++cc) {
            const int col = cb * 16 + cc;
            float h, l;
            fold4(vv[0][cc], vv[1][cc], vv[2][cc], vv[3][cc], h, l);
            store_out(a, col_dst[col], row, h, l, era + col_e[col], 0.0);
          }
        } else if (row_ok && a.out_mode != 2) {
#pragma unroll
          for (int cc = 0; cc < 16; ++cc) {
            const int col = cb * 16 + cc;
            if (col >= tile.ncol) break;
            float h, l;
            fold4(vv[0][cc], vv[1][cc], vv[2][cc], vv[3][cc], h, l);
            store_out(a, col_dst[col], row, h, l, era + col_e[col], 0.0);
          }
        } else if (row_ok) {
          // accumulating launch: fold first (the accumulators' registers are free again), then read
          // the old values of eight columns together, then store them
#pragma unroll
          for (int cc = 0; cc < 16; ++cc) {
            float h, l;
            fold4(vv[0][cc], vv[1][cc], vv[2][cc], vv[3][cc], h, l);
            vv[0][cc] = h;
            vv[1][cc] = l;
          }
#pragma unroll
          for (int c8 = 0; c8 < 16; c8 += 8) {
            double old[8];
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
              const int col = cb * 16 + c8 + cc;
              old[cc] = col < tile.ncol ? reinterpret_cast<const double*>(a.Y)[col_dst[col] + row] : 0.0;
            }
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
              const int col = cb * 16 + c8 + cc;
              if (col < tile.ncol)
                store_out(a, col_dst[col], row, vv[0][c8 + cc], vv[1][c8 + cc], era + col_e[col], old[cc]);
            }
          }
        }
      }
      // accumulators read: the MMA warp may start the next tile
      asm volatile("tcgen05.fence::before_thread_sync;\n");
      mbar_arrive(&tmem_free[buf]);
      // column metadata of this tile no longer needed by any epilogue thread
      asm volatile("bar.sync 1, %0;\n" ::"n"(kTcEpilogue) : "memory");
    }
    }
  } else if (lane == 0) {
    // ---- MMA issuer
    // instruction descriptor: D f32, A and B bf16, both K-major, M = 128, N = BN (TR for transposed
    // tiles)
    constexpr int kN = TR ? TR : BN;
    const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(kN >> 3) << 17) |
                           ((unsigned)(kSplitBM >> 4) << 24);
    // shared-memory descriptors of stage 0, slice 0; the start address (16-byte units, low bits) of
    // any other slice tile is an added constant, so a K step issues its S(S+1)/2 MMAs from
    // precomputed descriptors with no per-MMA arithmetic beyond one add (the single issuing thread
    // is the limit of the MMA rate otherwise).
    // A (tiled layout): next core matrix along K 2048 bytes further, next 8-row group 128 bytes
    const unsigned long long dA0 = umma_desc(smem_u32(As), 2048, 128);
    const unsigned long long dB0 = umma_desc(smem_u32(Bs), 128, 256);
    long long g = 0;
    bool ok = true;
    int it = 0;
    for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++it) {
      // the accumulator set of this tile is free once the epilogue has drained its previous use
      const int buf = it % kBufs;
      if (it >= kBufs && !mbar_wait(&tmem_free[buf], (unsigned)(it / kBufs - 1) & 1u, &abort_sh)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      for (int k = 0; k < nk; ++k, ++g) {
        const int st = (int)(g % kTcStages);
        if (!mbar_wait(&full[st], (unsigned)(g / kTcStages) & 1u, &abort_sh) ||
            !mbar_wait(&fullA[st], (unsigned)(g / kTcStages) & 1u, &abort_sh)) {
          ok = false;
          break;
        }
        // the B part of the stage was written through the generic proxy (cp.async); the MMA reads
        // it through the async proxy
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        const unsigned long long da = dA0 + (unsigned long long)((st * S * kTcA * 2) >> 4);
        const unsigned long long db = dB0 + (unsigned long long)((st * S * kTcB * 2) >> 4);
        // the first product of each accumulator in a tile (step 0, i = 0, j = w) overwrites it
        const unsigned acc = tmem + (unsigned)(buf * kAccCols);
        constexpr int kSA = (kSplitBM * 16 * 2) >> 4, kSB = (BN * 16 * 2) >> 4;  // slice tile strides
        if constexpr (TR > 0) {
          // gathered vectors as A (128 rows), operator slices as B (its first TR rows)
          if (k == 0) mma_kstep<S, TR, kSB, kSA, true>(acc, db, da, idesc);
          else mma_kstep<S, TR, kSB, kSA, false>(acc, db, da, idesc);
        } else {
          if (k == 0) mma_kstep<S, BN, kSA, kSB, true>(acc, da, db, idesc);
          else mma_kstep<S, BN, kSA, kSB, false>(acc, da, db, idesc);
        }
        umma_commit(&empty[st]);
      }
      if (ok) umma_commit(&accbar[buf]);
    }
    if (!ok) abort_sh = 1;
    // every MMA issued above has completed once this arrives
    umma_commit(&donebar);
    mbar_wait(&donebar, 0);
  }

  __syncthreads();
  if (tid == 0 && abort_sh) atomicExch(&g_split_error, 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == kTcMmaWarp) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(kTcCols));
  }
}

size_t tc_smem_bytes(int S, int BN) { return (size_t)kTcStages * S * (kTcA + BN * kTcKC) * sizeof(slice_t); }

// ------------------------------------------------------------------ reduction

// Reduction of double-float slots: y[dst] = sum of slots (double-float), written as FP64.
__global__ void k_reduce_df(DFReduceArgs a) {
  constexpr int kChunk = 64;  // slot offsets staged in shared memory per pass
  __shared__ long long slot_sh[kChunk];
  const int d = blockIdx.x;
  const long long b = a.ptr[d], e = a.ptr[d + 1];
  const float2* S = reinterpret_cast<const float2*>(a.S);
  const int rows_per_pass = (a.M + blockDim.x - 1) / blockDim.x;
  // each thread owns up to 4 rows (M <= 4 * blockDim.x), summed in slot order
  float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
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
      for (; k + 4 <= nc; k += 4) {  // four loads in flight, added in slot order
        const float2 v0 = S[slot_sh[k] + r], v1 = S[slot_sh[k + 1] + r];
        const float2 v2 = S[slot_sh[k + 2] + r], v3 = S[slot_sh[k + 3] + r];
        df_add(hi[q], lo[q], v0.x); df_add(hi[q], lo[q], v0.y);
        df_add(hi[q], lo[q], v1.x); df_add(hi[q], lo[q], v1.y);
        df_add(hi[q], lo[q], v2.x); df_add(hi[q], lo[q], v2.y);
        df_add(hi[q], lo[q], v3.x); df_add(hi[q], lo[q], v3.y);
      }
      for (; k < nc; ++k) {
        const float2 v = S[slot_sh[k] + r];
        df_add(hi[q], lo[q], v.x);
        df_add(hi[q], lo[q], v.y);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = threadIdx.x + q * blockDim.x;
    if (q >= rows_per_pass || r >= a.M) break;
    const double s = (double)hi[q] + (double)lo[q];
    if (a.final_out) {
      const int f = r / a.n, t = r - f * a.n;
      const long long o = a.dst_off[d] + t;
      if (f == 0) a.u[o] = s;
      else a.g[(f - 1) * a.N + o] = s;
    } else {
      a.Y[a.dst_off[d] + r] = s;
    }
  }
}

constexpr int kKAlign = 32;  // padded K: a multiple of both engines' K steps
int kpad(int K) { return (K + kKAlign - 1) / kKAlign * kKAlign; }

int slice_table(const double* A, int nmat, int M, int K, int lda, long long mstride, int S, SplitTable* out,
                cudaStream_t s) {
  out->M = M; out->K = K; out->Kpad = kpad(K); out->nmat = nmat; out->nrt = (M + kSplitBM - 1) / kSplitBM;
  const size_t nh = (size_t)nmat * out->nrt * kSplitBM * S * out->Kpad;
  TRY(cudaMalloc(&out->A, nh * sizeof(slice_t)));
  TRY(cudaMemsetAsync(out->A, 0, nh * sizeof(slice_t), s));  // rows past M stay zero
  TRY(cudaMalloc(&out->ea, (size_t)nmat * M * sizeof(int)));
  const long long rows = (long long)nmat * M;
  k_slice_rows<kSplitSlices><<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(
      A, mstride, lda, M, K, out->Kpad, nmat, out->nrt, (slice_t*)out->A, out->ea);
  TRY(cudaGetLastError());
  return VP_OK;
}

}  // namespace

int build_split(vp_tables_s* T, cudaStream_t s) {
  const int S = kSplitSlices;
  T->n_slices = S;
  auto* st = new (std::nothrow) SplitTables();
  if (!st) return VP_ERR_OOM;
  T->near_split = st;
  const int n = T->n, C = T->C, E = T->E, nl = T->levels + 1;
  if (n > kSplitKMax || E > kSplitKMax || 2 * C > kSplitKMax) return VP_ERR_ARG;
  int rc;
  if ((rc = slice_table(T->near, nl * kNearPos, 3 * n, n, n, (long long)3 * n * n, S, &st->near, s))) return rc;
  if ((rc = slice_table(T->s2m, nl, E, n, n, (long long)E * n, S, &st->s2m, s))) return rc;
  if ((rc = slice_table(T->l2t, nl, 3 * n, E, E, (long long)3 * n * E, S, &st->l2t, s))) return rc;
  if ((rc = slice_table(T->m2l, nl * kVOff * T->nch, C, C, C, (long long)C * C, S, &st->m2l, s))) return rc;
  if ((rc = slice_table(T->m2t, nl * kWPos * T->nch, 3 * n, C, C, (long long)3 * n * C, S, &st->m2t, s))) return rc;
  if ((rc = slice_table(T->s2l, nl * kXPos * T->nch, C, n, n, (long long)C * n, S, &st->s2l, s))) return rc;
  if ((rc = slice_table(T->m2m, nl * T->nch, C, 2 * C, 4 * C, (long long)C * 4 * C, S, &st->m2m_lo, s))) return rc;
  if ((rc = slice_table(T->m2m + 2 * C, nl * T->nch, C, 2 * C, 4 * C, (long long)C * 4 * C, S, &st->m2m_hi, s)))
    return rc;
  if ((rc = slice_table(T->l2l, nl * 4 * T->nch, C, C, C, (long long)C * C, S, &st->l2l, s))) return rc;
  TRY(cudaStreamSynchronize(s));
  return VP_OK;
}

void free_split_tables(vp_tables_s* T) {
  auto* st = static_cast<SplitTables*>(T->near_split);
  if (!st) return;
  for (SplitTable* t : {&st->near, &st->s2m, &st->l2t, &st->m2l, &st->m2t, &st->s2l, &st->m2m_lo, &st->m2m_hi,
                        &st->l2l}) {
    if (t->A) cudaFree(t->A);
    if (t->ea) cudaFree(t->ea);
  }
  delete st;
  T->near_split = nullptr;
}

// Persistent tcgen05 grid: one CTA per SM of the device last prepared.
int g_num_sms = 152;

// Per device: allow the GEMM kernels their dynamic shared memory (call outside stream capture).
int prepare_split_launch() {
  int dev = 0;
  TRY(cudaGetDevice(&dev));
  static bool done[64] = {false};
  if (dev >= 0 && dev < 64 && done[dev]) return VP_OK;
  TRY(cudaFuncSetAttribute(k_split_gemm<kSplitSlices, 128, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)mma_smem_bytes(kSplitSlices, 128, 64)));
  TRY(cudaFuncSetAttribute(k_split_gemm<kSplitSlices, 64, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)mma_smem_bytes(kSplitSlices, 64, 32)));
  TRY(cudaFuncSetAttribute(k_split_gemm_tc<kSplitSlices, 128, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc_smem_bytes(kSplitSlices, 128)));
  TRY(cudaFuncSetAttribute(k_split_gemm_tc<kSplitSlices, 64, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc_smem_bytes(kSplitSlices, 64)));
  TRY(cudaFuncSetAttribute(k_split_gemm_tc<kSplitSlices, 128, 96>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc_smem_bytes(kSplitSlices, 128)));
  TRY(cudaFuncSetAttribute(k_split_gemm_tc<kSplitSlices, 128, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc_smem_bytes(kSplitSlices, 128)));
  int sms = 0;
  TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  g_num_sms = sms > 0 ? sms : 1;
  if (dev >= 0 && dev < 64) done[dev] = true;
  return VP_OK;
}

int selftest_wait(long long budget, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(budget);
  TRY(cudaGetLastError());
  TRY(cudaStreamSynchronize(s));
  return VP_OK;
}

int read_split_error(int* flag) {
  int h = 0;
  TRY(cudaMemcpyFromSymbol(&h, g_split_error, sizeof(int)));
  const int zero = 0;
  TRY(cudaMemcpyToSymbol(g_split_error, &zero, sizeof(int)));
  *flag = h;
  return VP_OK;
}

int launch_split_gemm(const SplitArgs& a, int n_tiles, cudaStream_t s, int engine, int short_ctas) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  TRY(cudaStreamIsCapturing(s, &cs));
  if (cs == cudaStreamCaptureStatusNone) {
    const int rc = prepare_split_launch();
    if (rc) return rc;
  }
  if (n_tiles <= 0) return VP_OK;
  // transposed tiles need an operator of at most 128 rows; taller ones run on the 128 x 128 engine
  if (engine == kEngineTcgen05T && a.M > 128) engine = kEngineTcgen05;
  if (engine == kEngineTcgen05 || engine == kEngineTcgen05N64 || engine == kEngineTcgen05T) {
    // short_ctas: two tiles per CTA (CTAs end often enough for the far-field chain's launches to find
    // SMs, and the per-CTA setup is paid half as often: 7.00 vs 7.17 ms per overlapped evaluation of
    // the full-size star, 7.07 with four)
    const int grid = short_ctas ? (n_tiles + 1) / 2 : (n_tiles < g_num_sms ? n_tiles : g_num_sms);
    if (engine == kEngineTcgen05)
      k_split_gemm_tc<kSplitSlices, 128, 0><<<grid, kTcThreads, tc_smem_bytes(kSplitSlices, 128), s>>>(a, n_tiles);
    else if (engine == kEngineTcgen05N64)
      k_split_gemm_tc<kSplitSlices, 64, 0><<<grid, kTcThreads, tc_smem_bytes(kSplitSlices, 64), s>>>(a, n_tiles);
    else if (a.M <= 96)
      k_split_gemm_tc<kSplitSlices, 128, 96><<<grid, kTcThreads, tc_smem_bytes(kSplitSlices, 128), s>>>(a, n_tiles);
    else
      k_split_gemm_tc<kSplitSlices, 128, 128><<<grid, kTcThreads, tc_smem_bytes(kSplitSlices, 128), s>>>(a, n_tiles);
  }
  else if (engine == kEngineMmaSmall)
    k_split_gemm<kSplitSlices, 64, 32><<<n_tiles, 64, mma_smem_bytes(kSplitSlices, 64, 32), s>>>(a);
  else
    k_split_gemm<kSplitSlices, 128, 64><<<n_tiles, 256, mma_smem_bytes(kSplitSlices, 128, 64), s>>>(a);
  TRY(cudaGetLastError());
  return VP_OK;
}

int launch_slice_list(const double* X, const long long* base, const long long* vid, long long nlist, int K, int kseg,
                      long long seg_stride, long long cstride, void* out, int* eb, cudaStream_t s) {
  if (nlist <= 0) return VP_OK;
  k_slice_list<kSplitSlices><<<(unsigned)((nlist * 32 + 255) / 256), 256, 0, s>>>(
      X, base, vid, nlist, K, kseg > 0 ? kseg : K, seg_stride, cstride, kpad(K), (slice_t*)out, eb);
  TRY(cudaGetLastError());
  return VP_OK;
}

int launch_reduce_df(const DFReduceArgs& a, int n_dst, cudaStream_t s) {
  if (n_dst <= 0) return VP_OK;
  const int threads = a.M >= 256 ? 256 : ((a.M + 31) / 32) * 32;
  if (a.M > 4 * threads) return VP_ERR_ARG;  // rows per thread are held in registers (3 p^2 <= 768)
  k_reduce_df<<<n_dst, threads, 0, s>>>(a);
  TRY(cudaGetLastError());
  return VP_OK;
}

int split_kpad(int K) { return kpad(K); }

}  // namespace vp
