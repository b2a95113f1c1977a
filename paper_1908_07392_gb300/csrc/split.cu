// Split-precision contractions on the tensor cores (VP_PREC_SPLIT).
//
// An FP64 product y = A x (A an operator table, x a coefficient or nodal
// vector) is computed from exact integer slices, in the manner of Ozaki's
// error-free splitting of matrix products (Ozaki, Ogita, Oishi and Rump,
// Numer. Algorithms 59, 2012):
//   * each row r of A is scaled by 2^-ea[r] (ea[r] = exponent of the row's
//     largest entry, so the scaled row lies in (-1, 1)) and cut into S slices
//     of 8-bit integers: A[r,k] = 2^ea[r] * sum_i a_i[r,k] 2^(-8i) + rounding
//     remainder below 2^(ea[r] - 8S - 1);
//   * each vector x likewise with one exponent eb per vector;
//   * the slices are stored exactly in fp16 (|a_1| <= 256, |a_i| <= 128 for
//     i >= 2), so every product a_i b_j is exact and the tensor cores' fp32
//     accumulation over K <= 256 terms stays below 2^24, i.e. exact, for the
//     leading weights i + j <= 3 (and within 2^-24 of its own weight beyond);
//   * products with the same i + j = d share the weight 2^(-8d), so they are
//     accumulated together in fp32 and folded into a double-float (hi, lo)
//     pair of fp32 numbers with error-free two-sums; the result is scaled by
//     2^(ea[r] + eb) exactly. Terms with i + j > S + 1 are dropped.
// The double-float results are stored in 8-byte slots and summed per target
// in double-float by the reduction; FP64 arithmetic is needed only when a
// result is written as an FP64 coefficient.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "plan.h"
#include "split.h"
#include "vp_internal.h"

namespace vp {

namespace {

#define TRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_last_cuda(e_); return e_ == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA; } } while (0)

// Balanced base-256 digits of |x| * 2^(8S - e) (|x| < 2^e), taken straight from the FP64 bit pattern
// with integer arithmetic: T = round(|x| 2^(8S-e)) < 2^(8S) (+1 from rounding), then the digits from the
// least significant up, each moved into [-128, 127] with a carry, the leading one in [0, 256]; the sign
// of x is applied to every digit. x = 2^e sum_i a_i 2^(-8i) up to 2^(e - 8S - 1). Digits are exact in fp16.
template <int S>
__device__ inline void digits(double x, int e, __half* out, size_t stride) {
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
  for (int i = 0; i < S; ++i) out[i * stride] = __int2half_rn(neg ? -dig[i] : dig[i]);
}

// Exponent e with |v| < 2^e for v = max |x| > 0 (0 for v = 0).
__device__ inline int exponent_of(double v) {
  int e = 0;
  if (v > 0.0) frexp(v, &e);
  return e;
}

// Slice rows of a batch of matrices: A[mat][r][k] (row stride lda, matrix stride mstride) ->
// out[mat][s][r][Kpad] (fp16), ea[mat][r]. One warp per row.
template <int S>
__global__ void k_slice_rows(const double* __restrict__ A, long long mstride, int lda, int M, int K, int Kpad,
                             int nmat, __half* __restrict__ out, int* __restrict__ ea) {
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
  __half* o = out + (mat * S * M + r) * (long long)Kpad;
  const size_t sstride = (size_t)M * Kpad;
  for (int k = lane; k < Kpad; k += 32) digits<S>(k < K ? a[k] : 0.0, e, o + k, sstride);
  if (lane == 0) ea[mat * M + r] = e;
}

// Slice a list of vectors. Vector v (v < nlist) has identifier id = vid ? vid[v] : v and elements
// x_k = X[b + (k / kseg) * seg_stride + k % kseg], k < K, b = base ? base[v] : v * cstride;
// output out[id][s][Kpad] and eb[id]. One warp per vector.
template <int S>
__global__ void k_slice_list(const double* __restrict__ X, const long long* __restrict__ base,
                             const long long* __restrict__ vid, long long nlist, int K, int kseg,
                             long long seg_stride, long long cstride, int Kpad, __half* __restrict__ out,
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
  __half* o = out + id * (long long)S * Kpad;
  for (int k = lane; k < Kpad; k += 32) {
    const int sg = k / kseg;
    digits<S>(k < K ? X[b + sg * seg_stride + (k - sg * kseg)] : 0.0, e, o + k, Kpad);
  }
  if (lane == 0) eb[id] = e;
}

// ------------------------------------------------------------------ tensor-core GEMM

constexpr int kSBM = 128, kSBN = 48, kSKC = 32, kSPitch = kSKC + 8;  // halves per smem row
constexpr int kWN = 24, kNT = kWN / 8;  // columns and n8 tiles per warp

__device__ inline void df_add(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  const float l = __fadd_rn(lo, err);
  const float t = __fadd_rn(s, l);
  lo = __fsub_rn(l, __fsub_rn(t, s));
  hi = t;
}

__device__ inline void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(n));
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ inline void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ inline void ldmatrix_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}

__device__ inline void ldmatrix_x2(unsigned& r0, unsigned& r1, const void* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}

__device__ inline void mma16816(float* c, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int S>
__global__ void __launch_bounds__(256) k_split_gemm(SplitArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __half* As = reinterpret_cast<__half*>(smem_raw);                       // [2][S][BM][pitch]
  __half* Bs = As + 2 * S * kSBM * kSPitch;                                 // [2][S][BN][pitch]
  const SplitTile tile = a.tiles[blockIdx.x];
  const long long mat = a.a_mat[tile.group];
  const __half* Ag = a.A + mat * (long long)S * a.M * a.Kpad;
  const int* ea = a.ea + mat * a.M;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 3, wn = warp >> 2;  // 4 warps along M (32 rows), 2 along N (24 columns)
  const int gid = lane >> 2, tig = lane & 3;

  auto load_chunk = [&](int buf, int k0) {
    // A: S slices x BM rows x KC halves = S*BM*4 16-byte pieces
    for (int e = tid; e < S * kSBM * 4; e += 256) {
      const int s = e / (kSBM * 4), rem = e % (kSBM * 4);
      const int r = rem >> 2, c = (rem & 3) * 8;
      const int gr = tile.m0 + r;
      const bool ok = gr < a.M;
      const __half* src = Ag + ((long long)s * a.M + (ok ? gr : 0)) * a.Kpad + k0 + c;
      cp_async16(As + ((buf * S + s) * kSBM + r) * kSPitch + c, src, ok);
    }
    for (int e = tid; e < S * kSBN * 4; e += 256) {
      const int s = e / (kSBN * 4), rem = e % (kSBN * 4);
      const int col = rem >> 2, c = (rem & 3) * 8;
      const bool ok = col < tile.ncol;
      const long long v = ok ? a.src_vec[tile.col0 + col] : 0;
      const __half* src = a.B + (v * S + s) * (long long)a.Kpad + k0 + c;
      cp_async16(Bs + ((buf * S + s) * kSBN + col) * kSPitch + c, src, ok);
    }
    cp_async_commit();
  };

  // one fp32 accumulator per weight 2^(-8d), d = i + j = 2..S+1, kept over the whole K: the sums of
  // integer products stay exact (below 2^24) for d <= 3 and are folded into double-float only at the end
  float acc[S][2][kNT][4];
#pragma unroll
  for (int d = 0; d < S; ++d)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < kNT; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[d][i][j][c] = 0.f;

  const int nchunks = a.Kpad / kSKC;
  load_chunk(0, 0);
  for (int ch = 0; ch < nchunks; ++ch) {
    const int buf = ch & 1;
    if (ch + 1 < nchunks) {
      load_chunk(buf ^ 1, (ch + 1) * kSKC);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kSKC / 16; ++ks) {
      // B fragments in two halves of the slices (register budget), each A slice loaded once per half
      constexpr int H = (S + 1) / 2;
#pragma unroll
      for (int jh = 0; jh < 2; ++jh) {
        unsigned bf[H][kNT][2];
#pragma unroll
        for (int jj = 0; jj < H; ++jj) {
          const int j = jh * H + jj;
          if (j >= S) break;
          const __half* Bb = Bs + ((buf * S + j) * kSBN + wn * kWN) * kSPitch;
          unsigned r0, r1, r2, r3;
          ldmatrix_x4(r0, r1, r2, r3,
                      Bb + ((lane & 7) + ((lane >> 4) << 3)) * kSPitch + ks * 16 + ((lane >> 3) & 1) * 8);
          bf[jj][0][0] = r0; bf[jj][0][1] = r1;
          bf[jj][1][0] = r2; bf[jj][1][1] = r3;
          ldmatrix_x2(bf[jj][2][0], bf[jj][2][1], Bb + (16 + (lane & 7)) * kSPitch + ks * 16 + ((lane >> 3) & 1) * 8);
        }
#pragma unroll
        for (int i = 0; i < S; ++i) {
          if (i + jh * H >= S) break;
          const __half* Ab = As + ((buf * S + i) * kSBM + wm * 32) * kSPitch;
          unsigned af[2][4];  // two m16 tiles
#pragma unroll
          for (int mt = 0; mt < 2; ++mt)
            ldmatrix_x4(af[mt][0], af[mt][1], af[mt][2], af[mt][3],
                        Ab + (mt * 16 + (lane & 15)) * kSPitch + ks * 16 + (lane >> 4) * 8);
#pragma unroll
          for (int jj = 0; jj < H; ++jj) {
            const int j = jh * H + jj;  // slice indices i+1, j+1: weight index d - 2 = i + j
            if (j >= S || i + j >= S) break;
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
              for (int nt = 0; nt < kNT; ++nt) mma16816(acc[i + j][mt][nt], af[mt], bf[jj][nt]);
          }
        }
      }
    }
    __syncthreads();
  }

  float hi[2][kNT][4], lo[2][kNT][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < kNT; ++nt)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float h = 0.f, l = 0.f;
#pragma unroll
        for (int d = 0; d < S; ++d) df_add(h, l, __fmul_rn(acc[d][mt][nt][c], __int_as_float((127 - 8 * (d + 2)) << 23)));
        hi[mt][nt][c] = h;
        lo[mt][nt][c] = l;
      }

  // epilogue: scale by 2^(ea[row] + eb[col]) and store
#pragma unroll
  for (int nt = 0; nt < kNT; ++nt)
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
      const int col = wn * kWN + nt * 8 + tig * 2 + cc;
      if (col >= tile.ncol) continue;
      const long long v = a.src_vec[tile.col0 + col];
      const int eb = a.eb[v];
      const long long dst = a.dst_off[tile.col0 + col];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
          const int row = tile.m0 + wm * 32 + mt * 16 + gid + rr * 8;
          if (row >= a.M) continue;
          const int e = ea[row] + eb;
          const float h = hi[mt][nt][rr * 2 + cc], l = lo[mt][nt][rr * 2 + cc];
          if (a.out_mode == 0) {
            float2 o;
            o.x = ldexpf(h, e);
            o.y = ldexpf(l, e);
            reinterpret_cast<float2*>(a.Y)[dst + row] = o;
          } else {
            const double val = ldexp((double)h + (double)l, e);
            double* y = reinterpret_cast<double*>(a.Y) + dst + row;
            *y = (a.out_mode == 2) ? *y + val : val;
          }
        }
    }
}

// Reduction of double-float slots: y[dst] = sum of slots (double-float), written as FP64.
__global__ void k_reduce_df(DFReduceArgs a) {
  const int d = blockIdx.x;
  const long long b = a.ptr[d], e = a.ptr[d + 1];
  const float2* S = reinterpret_cast<const float2*>(a.S);
  for (int r = threadIdx.x; r < a.M; r += blockDim.x) {
    float hi = 0.f, lo = 0.f;
    for (long long k = b; k < e; ++k) {
      const float2 v = S[a.slot[k] + r];
      df_add(hi, lo, v.x);
      df_add(hi, lo, v.y);
    }
    const double s = (double)hi + (double)lo;
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

int kpad(int K) { return (K + kSKC - 1) / kSKC * kSKC; }

int slice_table(const double* A, int nmat, int M, int K, int lda, long long mstride, int S, SplitTable* out,
                cudaStream_t s) {
  out->M = M; out->K = K; out->Kpad = kpad(K); out->nmat = nmat;
  const size_t nh = (size_t)nmat * S * M * out->Kpad;
  TRY(cudaMalloc(&out->A, nh * sizeof(__half)));
  TRY(cudaMalloc(&out->ea, (size_t)nmat * M * sizeof(int)));
  const long long rows = (long long)nmat * M;
  k_slice_rows<kSplitSlices><<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(A, mstride, lda, M, K, out->Kpad,
                                                                                 nmat, (__half*)out->A, out->ea);
  TRY(cudaGetLastError());
  return VP_OK;
}

size_t split_smem_bytes(int S) { return (size_t)2 * S * (kSBM + kSBN) * kSPitch * sizeof(__half); }

}  // namespace

int build_split(vp_tables_s* T, cudaStream_t s) {
  const int S = kSplitSlices;
  T->n_slices = S;
  auto* st = new (std::nothrow) SplitTables();
  if (!st) return VP_ERR_OOM;
  T->near_split = st;
  const int n = T->n, C = T->C, E = T->E, nl = T->levels + 1;
  int rc;
  if ((rc = slice_table(T->near, nl * kNearPos, 3 * n, n, n, (long long)3 * n * n, S, &st->near, s))) return rc;
  if ((rc = slice_table(T->s2m, nl, E, n, n, (long long)E * n, S, &st->s2m, s))) return rc;
  if ((rc = slice_table(T->l2t, nl, 3 * n, E, E, (long long)3 * n * E, S, &st->l2t, s))) return rc;
  if ((rc = slice_table(T->m2l, nl * kVOff * T->nch, C, C, C, (long long)C * C, S, &st->m2l, s))) return rc;
  if ((rc = slice_table(T->m2t, nl * kWPos * T->nch, 3 * n, C, C, (long long)3 * n * C, S, &st->m2t, s))) return rc;
  if ((rc = slice_table(T->s2l, nl * kXPos * T->nch, C, n, n, (long long)C * n, S, &st->s2l, s))) return rc;
  if ((rc = slice_table(T->m2m, nl * T->nch, C, 4 * C, 4 * C, (long long)C * 4 * C, S, &st->m2m, s))) return rc;
  if ((rc = slice_table(T->l2l, nl * 4 * T->nch, C, C, C, (long long)C * C, S, &st->l2l, s))) return rc;
  TRY(cudaStreamSynchronize(s));
  return VP_OK;
}

void free_split_tables(vp_tables_s* T) {
  auto* st = static_cast<SplitTables*>(T->near_split);
  if (!st) return;
  for (SplitTable* t : {&st->near, &st->s2m, &st->l2t, &st->m2l, &st->m2t, &st->s2l, &st->m2m, &st->l2l}) {
    if (t->A) cudaFree(t->A);
    if (t->ea) cudaFree(t->ea);
  }
  delete st;
  T->near_split = nullptr;
}

// Per device: allow the GEMM kernel its dynamic shared memory (call outside stream capture).
int prepare_split_launch() {
  int dev = 0;
  TRY(cudaGetDevice(&dev));
  static bool done[64] = {false};
  if (dev >= 0 && dev < 64 && done[dev]) return VP_OK;
  TRY(cudaFuncSetAttribute(k_split_gemm<kSplitSlices>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)split_smem_bytes(kSplitSlices)));
  if (dev >= 0 && dev < 64) done[dev] = true;
  return VP_OK;
}

int launch_split_gemm(const SplitArgs& a, int n_tiles, cudaStream_t s) {
  const size_t smem = split_smem_bytes(kSplitSlices);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  TRY(cudaStreamIsCapturing(s, &cs));
  if (cs == cudaStreamCaptureStatusNone) {
    const int rc = prepare_split_launch();
    if (rc) return rc;
  }
  if (n_tiles <= 0) return VP_OK;
  k_split_gemm<kSplitSlices><<<n_tiles, 256, smem, s>>>(a);
  TRY(cudaGetLastError());
  return VP_OK;
}

int launch_slice_list(const double* X, const long long* base, const long long* vid, long long nlist, int K, int kseg,
                      long long seg_stride, long long cstride, void* out, int* eb, cudaStream_t s) {
  if (nlist <= 0) return VP_OK;
  k_slice_list<kSplitSlices><<<(unsigned)((nlist * 32 + 255) / 256), 256, 0, s>>>(
      X, base, vid, nlist, K, kseg > 0 ? kseg : K, seg_stride, cstride, kpad(K), (__half*)out, eb);
  TRY(cudaGetLastError());
  return VP_OK;
}

int launch_reduce_df(const DFReduceArgs& a, int n_dst, cudaStream_t s) {
  if (n_dst <= 0) return VP_OK;
  const int threads = a.M >= 256 ? 256 : ((a.M + 31) / 32) * 32;
  k_reduce_df<<<n_dst, threads, 0, s>>>(a);
  TRY(cudaGetLastError());
  return VP_OK;
}

int split_kpad(int K) { return kpad(K); }

}  // namespace vp
