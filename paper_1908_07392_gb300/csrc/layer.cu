// Layer potential on the volume tree: the operators that connect boundary point sources to the
// tree's expansions and nodes.
//
// u^H = D[mu] (Sec. 2.2, Eqs. uH_dbl, dbl_lyr_pot, discretised by the boundary quadrature of
// Eq. dbl_lyr_quad) is a sum of point sources on the boundary. Each velocity component solves
// Laplacian (alpha^2 - Laplacian) u = 0 away from them, so the far field is represented in the same
// two-channel bases as the modified-biharmonic volume potential (Sec. 3.2.1, Eqs. mpole and loc:
// K_m(alpha rho) and log rho, rho^-m outside a box; I_m(alpha rho) and rho^m inside), and the
// tree's translation and target operators apply unchanged. The kernel is split by channel
// (dl_kernel_split: Bessel terms are derivatives of K0, algebraic terms derivatives of log r).
//
//  * multipole coefficients of a source (kind 0): the channel fields sampled at Q points on a circle
//    of radius R = 1.25 r about the box centre (r the box circumradius; every source lies within
//    r), Fourier coefficients by a discrete transform, divided by the basis values on that circle
//    (K_m(alpha R) / K_m(alpha r), (r/R)^m). Modes decay like (r/R)^m, so Q = 256 samples leave no
//    aliasing at order P <= 60. The log coefficient of channel L is the total charge of the
//    source, zero for the derivatives of log r that make up the double layer, and is set so.
//  * local coefficients (kind 1, the X lists): the fields sampled on the target box's circumcircle,
//    where the local basis functions are cos(m theta), sin(m theta).
//  * near values: the full kernel at the target leaf's nodes (the plain boundary quadrature).
// The paper forms the same expansions analytically from dipole and octopole moments (Eqs. dipole,
// quadrupole, octopole) and the addition theorems; sampling reaches the same coefficients to
// rounding and needs no per-moment formulas.
#include <cuda_runtime.h>

#include "layer.h"
#include "special.cuh"
#include "stokes.cuh"
#include "vp_internal.h"

namespace vp {

namespace {

#define TRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_last_cuda(e_); return e_ == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA; } } while (0)

constexpr int kQ = 256;       // samples on the circle
constexpr int kMaxP = 60;     // highest expansion order

__global__ void __launch_bounds__(kQ) k_pt_coeffs(int kind, double alpha, int P, const PtInst* inst, PtSources S,
                                                    double* A) {
  const PtInst I = inst[blockIdx.x];
  const int j = blockIdx.y;
  if (j >= I.ns) return;  // uniform over the block
  __shared__ double F[2][4][kQ];
  __shared__ double cq[kQ], sq[kQ];
  __shared__ double scl[2][kMaxP + 1];
  const int q = threadIdx.x;
  const int src = S.perm[I.j0 + j];
  const double yx = S.x[src], yy = S.y[src], nx = S.nx[src], ny = S.ny[src], w = S.w[src];
  {
    double sn, cs;
    sincospi(2.0 * q / kQ, &sn, &cs);
    cq[q] = cs;
    sq[q] = sn;
    double DK[4], DL[4];
    dl_kernel_split(alpha, I.cx + I.R * cs - yx, I.cy + I.R * sn - yy, nx, ny, DK, DL);
    for (int k = 0; k < 4; ++k) {
      F[0][k][q] = DK[k] * w;
      F[1][k][q] = DL[k] * w;
    }
  }
  if (q == 0) {
    if (kind == 0) {
      // K_m(alpha r) / K_m(alpha R) = [Khat_m(alpha r) / Khat_m(alpha R)] (R/r)^m, Khat scaled by e^z
      double kr[kMaxP + 2], kR[kMaxP + 2];
      khat_scaled(alpha * I.r, P + 1, kr);
      khat_scaled(alpha * I.R, P + 1, kR);
      const double ex = exp(alpha * (I.R - I.r));
      double pw = 1.0;
      for (int m = 0; m <= P; ++m) {
        scl[0][m] = I.kact ? kr[m] / kR[m] * ex * pw : 0.0;
        scl[1][m] = (m == 0) ? 0.0 : pw;
        pw *= I.R / I.r;
      }
    } else {
      for (int m = 0; m <= P; ++m) {
        scl[0][m] = I.kact ? 1.0 : 0.0;
        scl[1][m] = 1.0;
      }
    }
  }
  __syncthreads();
  const int C = 2 * P + 1, E = 2 * C;
  const int rows = 2 * E;
  for (int o = threadIdx.x; o < 4 * E; o += blockDim.x) {
    const int b = o & 1;
    int t = o >> 1;  // a E + ch C + mode
    const int mode = t % C;
    const int ch = (t / C) % 2, a = t / E;
    const int m = mode <= P ? mode : mode - P;
    const double* f = F[ch][2 * a + b];
    const double* tr = mode <= P ? cq : sq;
    double acc = 0.0;
    int idx = 0;
    for (int qq = 0; qq < kQ; ++qq) {
      acc = fma(f[qq], tr[idx], acc);
      idx += m;
      if (idx >= kQ) idx -= kQ;
    }
    acc *= (m == 0 ? 1.0 : 2.0) / kQ;
    A[I.aoff + (long long)(2 * j + b) * rows + t] = acc * scl[ch][m];
  }
}

__global__ void __launch_bounds__(256) k_pt_near(double alpha, int p, const double* xi, const PtInst* inst,
                                                  PtSources S, double* A) {
  const PtInst I = inst[blockIdx.x];
  const int n = p * p;
  const int i = threadIdx.x;
  if (i >= n) return;
  const double h = I.R;
  const double x = I.cx + 0.5 * (1.0 + xi[i % p]) * h, y = I.cy + 0.5 * (1.0 + xi[i / p]) * h;
  const int rows = 2 * n;
  for (int j = 0; j < I.ns; ++j) {
    const int src = S.perm[I.j0 + j];
    const double rx = x - S.x[src], ry = y - S.y[src];
    double D[4] = {0.0, 0.0, 0.0, 0.0};
    if (rx != 0.0 || ry != 0.0) dl_kernel(alpha, rx, ry, S.nx[src], S.ny[src], D);
    const double w = S.w[src];
    for (int b = 0; b < 2; ++b) {
      double* col = A + I.aoff + (long long)(2 * j + b) * rows;
      col[i] = D[b] * w;          // row a = 0
      col[n + i] = D[2 + b] * w;  // row a = 1
    }
  }
}

constexpr int kApplyThreads = 256, kApplyRows = 4, kApplyChunk = 1024;

__global__ void __launch_bounds__(kApplyThreads) k_pt_apply(int rows, int rb, long long bs, int df,
                                                             const PtInst* inst, const int* perm, const double* mu,
                                                             const double* A, double* Y) {
  __shared__ double xs[kApplyChunk];
  const PtInst I = inst[blockIdx.x];
  const int K = 2 * I.ns;
  double acc[kApplyRows] = {0.0, 0.0, 0.0, 0.0};
  for (int k0 = 0; k0 < K; k0 += kApplyChunk) {
    const int kc = min(kApplyChunk, K - k0);
    __syncthreads();
    for (int k = threadIdx.x; k < kc; k += kApplyThreads) {
      const int jj = (k0 + k) >> 1, b = (k0 + k) & 1;
      xs[k] = mu[2 * (long long)perm[I.j0 + jj] + b];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kApplyRows; ++q) {
      const int r = threadIdx.x + q * kApplyThreads;
      if (r >= rows) break;
      const double* a = A + I.aoff + (long long)k0 * rows + r;
      double s = acc[q];
      for (int k = 0; k < kc; ++k) s = fma(a[(long long)k * rows], xs[k], s);
      acc[q] = s;
    }
  }
#pragma unroll
  for (int q = 0; q < kApplyRows; ++q) {
    const int r = threadIdx.x + q * kApplyThreads;
    if (r >= rows) break;
    const long long o = I.dst + (long long)(r / rb) * bs + r % rb;
    if (df) {
      // double-float slot (the contribution slots of split-precision trees): high and low fp32 parts
      const float h = __double2float_rn(acc[q]);
      reinterpret_cast<float2*>(Y)[o] = make_float2(h, __double2float_rn(acc[q] - (double)h));
    } else {
      Y[o] = acc[q];
    }
  }
}

}  // namespace

int launch_pt_coeffs(int kind, double alpha, int P, const PtInst* inst, int n_inst, int max_ns, PtSources src,
                     double* A, cudaStream_t s) {
  if (n_inst <= 0 || max_ns <= 0) return VP_OK;
  if (P > kMaxP || max_ns > 65535) return VP_ERR_ARG;
  k_pt_coeffs<<<dim3((unsigned)n_inst, (unsigned)max_ns), kQ, 0, s>>>(kind, alpha, P, inst, src, A);
  TRY(cudaGetLastError());
  return VP_OK;
}

int launch_pt_near(double alpha, int p, const double* xi, const PtInst* inst, int n_inst, int max_ns,
                   PtSources src, double* A, cudaStream_t s) {
  (void)max_ns;
  if (n_inst <= 0) return VP_OK;
  if (p * p > 256) return VP_ERR_ARG;
  k_pt_near<<<(unsigned)n_inst, 256, 0, s>>>(alpha, p, xi, inst, src, A);
  TRY(cudaGetLastError());
  return VP_OK;
}

int launch_pt_apply(int rows, int rb, long long bs, int df, const PtInst* inst, int n_inst, const int* perm,
                    const double* mu, const double* A, double* Y, cudaStream_t s) {
  if (n_inst <= 0) return VP_OK;
  if (rows > kApplyThreads * kApplyRows || rb <= 0) return VP_ERR_ARG;
  k_pt_apply<<<(unsigned)n_inst, kApplyThreads, 0, s>>>(rows, rb, bs, df, inst, perm, mu, A, Y);
  TRY(cudaGetLastError());
  return VP_OK;
}

}  // namespace vp
