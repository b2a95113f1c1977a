// Periodic particular solution by FFT (Sec. 2.1, Eqs. uhat, periodic_stokeslet, uP_Fourier,
// uP_Fourier_deriv; Sec. 3.1.2): on a uniform n x n grid of the periodic box of side L, the velocity
// of the modified Stokes equations (alpha^2 - Laplacian) u + grad p = F, div u = 0 is
//   u_hat(k) = S_hat(k) F_hat(k),  S_hat = (I - k k^T / |k|^2) / (alpha^2 + |k|^2),  S_hat(0) = I / alpha^2,
// and its gradient is i k_m u_hat. This is the paper's own route to the particular solution (the
// force extended by PUX, which stays out of scope here; the caller supplies the periodic force).
//
// Transforms: complex FP64, n a power of two (16 .. 4096), radix-2 Stockham autosort (natural order
// in and out, no bit reversal) on rows held in shared memory, rows then columns through a tiled
// transpose. Real fields travel in pairs as the real and imaginary parts of one complex field: the
// forward transform of F_x + i F_y gives both spectra (split by conjugate symmetry), and three
// inverse transforms give (u_x, u_y), (du_x/dx, du_x/dy), (du_y/dx, du_y/dy). On this GPU the FP64
// pipe, not memory, bounds the butterflies.
#include <cuda_runtime.h>

#include <cmath>
#include <new>
#include <vector>

#include "special.cuh"
#include "vp_internal.h"

struct vp_periodic_s {
  double alpha = 0.0, side = 0.0;
  int n = 0, logn = 0;
  double2* tw_f = nullptr;  // e^{-2 pi i q / n}, q < n
  double2* tw_i = nullptr;  // e^{+2 pi i q / n}
  double2* a = nullptr;     // work arrays [n][n]
  double2* b = nullptr;
  double2* c = nullptr;
  double2* d = nullptr;
};

namespace vp {
namespace {

#define TRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_last_cuda(e_); return e_ == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA; } } while (0)

constexpr int kFftThreads = 512;
constexpr int kMaxN = 4096;

__device__ inline double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// One length-n transform per block (row blockIdx.x of data [rows][n]), in place, unnormalised: Stockham
// autosort, decimation in frequency, radix 4 (and one radix-2 stage when log2 n is odd), ping-pong in
// shared memory. A stage of radix r with m points already combined (l = n / (r m)) maps, for j < l and
// k < m, the inputs a_q = x[k + (j + q l) m] (q < r) to
//   y[k + (r j + p) m] = w^(p j m) b_p,   b_p = sum_q a_q e^(-+2 pi i p q / r),   w = e^(-+2 pi i / n),
// then m *= r. `dir` is the sign of the exponent (-1 forward, +1 inverse) and tw[q] = e^(dir 2 pi i q / n).
__device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

__global__ void __launch_bounds__(kFftThreads) k_fft_rows(int n, int logn, int dir, double2* data, const double2* tw) {
  extern __shared__ double2 fsm[];
  double2* x = fsm;
  double2* y = fsm + n;
  double2* row = data + (size_t)blockIdx.x * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = row[i];
  __syncthreads();
  int lg_m = 0;  // log2 m
  if (logn & 1) {
    // radix-2 stage first (m = 1, l = n / 2): twiddle index p j m = j for p = 1
    const int l = n >> 1;
    for (int j = threadIdx.x; j < l; j += blockDim.x) {
      const double2 a0 = x[j], a1 = x[j + l];
      y[2 * j] = cadd(a0, a1);
      y[2 * j + 1] = cmul(tw[j], csub(a0, a1));
    }
    __syncthreads();
    double2* t = x; x = y; y = t;
    lg_m = 1;
  }
  for (; lg_m < logn; lg_m += 2) {
    const int m = 1 << lg_m, lg_l = logn - 2 - lg_m, l = 1 << lg_l;
    for (int idx = threadIdx.x; idx < (n >> 2); idx += blockDim.x) {
      const int j = idx >> lg_m, k = idx & (m - 1);
      const int i0 = k + j * m, lm = l * m;
      const double2 a0 = x[i0], a1 = x[i0 + lm], a2 = x[i0 + 2 * lm], a3 = x[i0 + 3 * lm];
      const double2 s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
      // e^(dir i pi / 2) (a1 - a3) = dir i d13
      const double2 r13 = make_double2(-dir * d13.y, dir * d13.x);
      const int o = k + 4 * j * m, jm = j * m;
      y[o] = cadd(s02, s13);
      y[o + m] = cmul(tw[jm], cadd(d02, r13));
      y[o + 2 * m] = cmul(tw[2 * jm], csub(s02, s13));
      y[o + 3 * m] = cmul(tw[3 * jm], csub(d02, r13));
    }
    __syncthreads();
    double2* t = x; x = y; y = t;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) row[i] = x[i];
}

// out[c][r] = in[r][c] for n x n complex, 32 x 32 tiles.
__global__ void k_transpose(int n, const double2* in, double2* out) {
  __shared__ double2 t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) t[j][threadIdx.x] = in[(size_t)(by + j) * n + bx + threadIdx.x];
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) out[(size_t)(bx + j) * n + by + threadIdx.x] = t[threadIdx.x][j];
}

__global__ void k_pack(long long nn, const double* fx, const double* fy, double2* z) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < nn) z[i] = make_double2(fx[i], fy[i]);
}

// Spectral step. Z = FFT(F_x + i F_y) in [ky][kx] order. F_x hat = (Z(k) + conj Z(-k)) / 2,
// F_y hat = (Z(k) - conj Z(-k)) / (2i). Writes A = u_x + i u_y, B = d_x u_x + i d_y u_x,
// C = d_x u_y + i d_y u_y in spectral space, scaled by 1/n^2 for the unnormalised inverse.
// The Nyquist wavenumber carries no derivative (its sine mode vanishes on the grid).
__global__ void k_spectral(int n, double alpha, double two_pi_over_L, const double2* Z, double2* A, double2* B,
                           double2* C) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)n * n) return;
  const int ix = (int)(i % n), iy = (int)(i / n);
  const int jx = (n - ix) & (n - 1), jy = (n - iy) & (n - 1);
  const double2 z = Z[i], zm = Z[(size_t)jy * n + jx];
  const double2 fx = make_double2(0.5 * (z.x + zm.x), 0.5 * (z.y - zm.y));
  const double2 fy = make_double2(0.5 * (z.y + zm.y), -0.5 * (z.x - zm.x));
  const int kxi = ix < n / 2 ? ix : ix - n, kyi = iy < n / 2 ? iy : iy - n;
  const double kx = two_pi_over_L * kxi, ky = two_pi_over_L * kyi;
  const double k2 = kx * kx + ky * ky;
  double2 ux, uy;
  if (k2 == 0.0) {
    ux = make_double2(fx.x / (alpha * alpha), fx.y / (alpha * alpha));
    uy = make_double2(fy.x / (alpha * alpha), fy.y / (alpha * alpha));
  } else {
    const double den = 1.0 / (k2 * (alpha * alpha + k2));
    // on the Nyquist row or column (not the corner) the wavenumber n/2 stands for +n/2 and -n/2 alike,
    // and the cross term, odd in it, averages to zero: the multiplier of a real field stays even
    const bool nyq_edge = (ix == n / 2) != (iy == n / 2);
    const double sxx = ky * ky * den, sxy = nyq_edge ? 0.0 : -kx * ky * den, syy = kx * kx * den;
    ux = make_double2(sxx * fx.x + sxy * fy.x, sxx * fx.y + sxy * fy.y);
    uy = make_double2(sxy * fx.x + syy * fy.x, sxy * fx.y + syy * fy.y);
  }
  const double dx = (ix == n / 2) ? 0.0 : kx, dy = (iy == n / 2) ? 0.0 : ky;
  const double sc = 1.0 / ((double)n * (double)n);
  // A = ux + i uy
  A[i] = make_double2(sc * (ux.x - uy.y), sc * (ux.y + uy.x));
  // B = i dx ux + i (i dy ux) = i ux (dx + i dy) ; C likewise with uy
  const double2 g = make_double2(-dy, dx);  // i (dx + i dy)
  B[i] = make_double2(sc * (g.x * ux.x - g.y * ux.y), sc * (g.x * ux.y + g.y * ux.x));
  C[i] = make_double2(sc * (g.x * uy.x - g.y * uy.y), sc * (g.x * uy.y + g.y * uy.x));
}

__global__ void k_unpack(long long nn, const double2* z, double* re, double* im) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const double2 v = z[i];
  re[i] = v.x;
  im[i] = v.y;
}

__global__ void k_twiddles(int n, double sign, double2* tw) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  double s, c;
  sincospi(2.0 * q / n, &s, &c);
  tw[q] = make_double2(c, sign * s);
}

size_t fft_smem(int n) { return (size_t)2 * n * sizeof(double2); }

// 2D transform of X [n][n] in place (rows, transpose into W, rows, transpose back).
int fft2d(const vp_periodic_s* P, double2* X, double2* W, const double2* tw, int dir, cudaStream_t s) {
  const int n = P->n;
  k_fft_rows<<<n, kFftThreads, fft_smem(n), s>>>(n, P->logn, dir, X, tw);
  TRY(cudaGetLastError());
  const dim3 tg(n / 32, n / 32), tb(32, 8);
  k_transpose<<<tg, tb, 0, s>>>(n, X, W);
  TRY(cudaGetLastError());
  k_fft_rows<<<n, kFftThreads, fft_smem(n), s>>>(n, P->logn, dir, W, tw);
  TRY(cudaGetLastError());
  k_transpose<<<tg, tb, 0, s>>>(n, W, X);
  TRY(cudaGetLastError());
  return VP_OK;
}

}  // namespace
}  // namespace vp

using namespace vp;

extern "C" int vp_periodic_create(double alpha, int n, double side, void* stream, vp_periodic* out) {
  if (!out) return VP_ERR_ARG;
  *out = nullptr;
  if (!(alpha > 0.0) || !(side > 0.0) || n < 32 || n > kMaxN || (n & (n - 1))) return VP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  vp_periodic_s* P = new (std::nothrow) vp_periodic_s();
  if (!P) return VP_ERR_OOM;
  P->alpha = alpha; P->side = side; P->n = n;
  while ((1 << P->logn) < n) ++P->logn;
  auto fail = [&](int code) { vp_periodic_free(P); return code; };
  const size_t nn = (size_t)n * n;
  for (double2** p : {&P->a, &P->b, &P->c, &P->d}) {
    if (cudaMalloc(p, nn * sizeof(double2)) != cudaSuccess) { cudaGetLastError(); return fail(VP_ERR_OOM); }
  }
  if (cudaMalloc(&P->tw_f, n * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(&P->tw_i, n * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    return fail(VP_ERR_OOM);
  }
  k_twiddles<<<(n + 255) / 256, 256, 0, s>>>(n, -1.0, P->tw_f);
  k_twiddles<<<(n + 255) / 256, 256, 0, s>>>(n, 1.0, P->tw_i);
  if (cudaFuncSetAttribute(k_fft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem(kMaxN)) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    set_last_cuda(cudaGetLastError());
    return fail(VP_ERR_CUDA);
  }
  *out = P;
  return VP_OK;
}

extern "C" int vp_periodic_eval(vp_periodic P, const double* F, double* u, double* gradu, void* stream) {
  if (!P || !F || !u || !gradu) return VP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n = P->n;
  const long long nn = (long long)n * n;
  const unsigned g = (unsigned)((nn + 255) / 256);
  k_pack<<<g, 256, 0, s>>>(nn, F, F + nn, P->a);
  TRY(cudaGetLastError());
  int rc = fft2d(P, P->a, P->b, P->tw_f, -1, s);
  if (rc) return rc;
  // spectra of (u_x + i u_y), (d_x u_x + i d_y u_x), (d_x u_y + i d_y u_y)
  k_spectral<<<g, 256, 0, s>>>(n, P->alpha, 2.0 * kPi / P->side, P->a, P->b, P->c, P->d);
  TRY(cudaGetLastError());
  for (int f = 0; f < 3; ++f) {
    double2* X = f == 0 ? P->b : (f == 1 ? P->c : P->d);
    if ((rc = fft2d(P, X, P->a, P->tw_i, 1, s))) return rc;
    double* re = f == 0 ? u : gradu + (size_t)(f - 1) * 2 * nn;
    double* im = f == 0 ? u + nn : re + nn;
    k_unpack<<<g, 256, 0, s>>>(nn, X, re, im);
    TRY(cudaGetLastError());
  }
  return VP_OK;
}

extern "C" void vp_periodic_free(vp_periodic P) {
  if (!P) return;
  for (void* p : {(void*)P->a, (void*)P->b, (void*)P->c, (void*)P->d, (void*)P->tw_f, (void*)P->tw_i})
    if (p) cudaFree(p);
  delete P;
}
