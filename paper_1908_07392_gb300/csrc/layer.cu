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

#include <algorithm>
#include <vector>

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

// ------------------------------------------------------------------------------------------------
// Near-boundary correction (Sec. 4.2, 4.4: the plain panel rule fails for targets within about a panel
// length of the panel; the paper corrects those point-panel pairs with precomputed weights).
//
// For a pair (target x, panel [ta, tb] of the parameter), the panel's contribution with the density
// interpolated by the panel's Lagrange basis in t,
//     int_panel D(x - y(t)) l_j(t) |y'(t)| dt,   j = 0 .. 15,
// is integrated on the exact curve by Gauss-Legendre (20 points) on pieces graded dyadically toward
// t0, the parameter of the closest point: each piece lies about its own length away from x, so the
// near-singular integrand is resolved at every distance, down to pieces shorter than half the distance
// d. The kernel is evaluated directly (App. B closed form, App. C series for small alpha r), so the
// panel needs no subdivision for large alpha h (the kernel-split quadrature of Sec. 4.2 needs alpha h
// <= 4.5, Eq. alpha_h_crit, because its split parts grow like e^(alpha r)). The plain weight
// D(x - y_j) w_j, which the tree sum already contains, is subtracted.
namespace vp {
namespace {

constexpr int kGQ = 20;        // Gauss-Legendre points per graded piece
constexpr int kMaxGrade = 44;  // dyadic levels per side at most
__constant__ double c_g20x[kGQ], c_g20w[kGQ], c_g16x[kNearQ], c_g16w[kNearQ], c_bw16n[kNearQ];

__device__ inline void star_point(const StarGeom& g, double t, double& x, double& y, double& sp) {
  double s, c, s5, c5;
  sincos(t, &s, &c);
  sincos(g.k * t + g.phase, &s5, &c5);
  const double r = g.R + g.A * c5, dr = -g.A * g.k * s5;
  x = r * c;
  y = r * s;
  const double dx = dr * c - r * s, dy = dr * s + r * c;
  sp = sqrt(dx * dx + dy * dy);
}

__device__ inline void star_normal(const StarGeom& g, double t, double& nx, double& ny) {
  double s, c, s5, c5;
  sincos(t, &s, &c);
  sincos(g.k * t + g.phase, &s5, &c5);
  const double r = g.R + g.A * c5, dr = -g.A * g.k * s5;
  const double dx = dr * c - r * s, dy = dr * s + r * c;
  const double sp = sqrt(dx * dx + dy * dy);
  nx = -dy / sp;  // counter-clockwise: the interior is on the left of the tangent
  ny = dx / sp;
}

// One 64-thread block per pair: in rounds of 64 quadrature points each thread evaluates the kernel
// and the 16 Lagrange basis values at one point into shared memory, then thread (j, ab) accumulates
// its weight over the round.
__global__ void __launch_bounds__(64) k_near_weights(double alpha, StarGeom g, const NearPair* pairs, double* dW) {
  __shared__ double Dq[64][4], Lq[64][kNearQ];
  const NearPair P = pairs[blockIdx.x];
  const double hp = 2.0 * kPi / g.n_panels;
  const double ta = P.panel * hp, tb = ta + hp;
  // graded pieces: left of t0 (toward t0 from ta) and right (toward t0 from tb); the length of
  // the last piece is below half the distance (arc length ~ parameter length times the speed)
  double x0, y0, sp0;
  star_point(g, P.t0, x0, y0, sp0);
  const double dmin = fmax(P.d, 1e-14 * hp * sp0);
  int nl = 0, nr = 0;
  if (P.t0 - ta > 0.0) {
    double len = P.t0 - ta;
    while (nl < kMaxGrade && len * sp0 > 0.5 * dmin) { len *= 0.5; ++nl; }
  }
  if (tb - P.t0 > 0.0) {
    double len = tb - P.t0;
    while (nr < kMaxGrade && len * sp0 > 0.5 * dmin) { len *= 0.5; ++nr; }
  }
  // pieces: left k = 0..nl-1: [t0 - L/2^k, t0 - L/2^(k+1)], then [t0 - L/2^nl, t0]; right likewise
  const int n_left = (P.t0 - ta > 0.0) ? nl + 1 : 0, n_right = (tb - P.t0 > 0.0) ? nr + 1 : 0;
  const int n_pts = (n_left + n_right) * kGQ;
  const int j = threadIdx.x >> 2, ab = threadIdx.x & 3;
  double acc = 0.0;
  for (int q0 = 0; q0 < n_pts; q0 += 64) {
    const int q = q0 + threadIdx.x;
    __syncthreads();
    if (q < n_pts) {
      const int piece = q / kGQ, m = q % kGQ;
      double a, b;
      if (piece < n_left) {
        const double L = P.t0 - ta;
        a = (piece < nl) ? P.t0 - L * ldexp(1.0, -piece) : P.t0 - L * ldexp(1.0, -nl);
        b = (piece < nl) ? P.t0 - L * ldexp(1.0, -piece - 1) : P.t0;
      } else {
        const int k = piece - n_left;
        const double L = tb - P.t0;
        a = (k < nr) ? P.t0 + L * ldexp(1.0, -k - 1) : P.t0;
        b = (k < nr) ? P.t0 + L * ldexp(1.0, -k) : P.t0 + L * ldexp(1.0, -nr);
      }
      const double t = 0.5 * (a + b) + 0.5 * (b - a) * c_g20x[m];
      const double wq = 0.5 * (b - a) * c_g20w[m];
      double yx, yy, sp, nx, ny;
      star_point(g, t, yx, yy, sp);
      star_normal(g, t, nx, ny);
      double D[4] = {0.0, 0.0, 0.0, 0.0};
      const double rx = P.x - yx, ry = P.y - yy;
      if (rx != 0.0 || ry != 0.0) dl_kernel(alpha, rx, ry, nx, ny, D);
      for (int c = 0; c < 4; ++c) Dq[threadIdx.x][c] = D[c] * wq * sp;
      // Lagrange basis of the panel's nodes at t (barycentric, reference coordinate in [-1, 1])
      const double tau = 2.0 * (t - ta) / hp - 1.0;
      double den = 0.0;
      int hit = -1;
      for (int i = 0; i < kNearQ; ++i) {
        const double dd = tau - c_g16x[i];
        if (dd == 0.0) hit = i;
        else den += c_bw16n[i] / dd;
      }
      for (int i = 0; i < kNearQ; ++i)
        Lq[threadIdx.x][i] = (hit >= 0) ? (i == hit ? 1.0 : 0.0) : (c_bw16n[i] / (tau - c_g16x[i])) / den;
    } else {
      for (int c = 0; c < 4; ++c) Dq[threadIdx.x][c] = 0.0;
      for (int i = 0; i < kNearQ; ++i) Lq[threadIdx.x][i] = 0.0;
    }
    __syncthreads();
    const int nq = min(64, n_pts - q0);
    for (int qq = 0; qq < nq; ++qq) acc = fma(Dq[qq][ab], Lq[qq][j], acc);
  }
  // minus the plain weight of node j: D(x - y_j) w_j
  {
    const double t = ta + 0.5 * hp * (1.0 + c_g16x[j]);
    double yx, yy, sp, nx, ny;
    star_point(g, t, yx, yy, sp);
    star_normal(g, t, nx, ny);
    double D[4] = {0.0, 0.0, 0.0, 0.0};
    const double rx = P.x - yx, ry = P.y - yy;
    if (rx != 0.0 || ry != 0.0) dl_kernel(alpha, rx, ry, nx, ny, D);
    acc -= D[ab] * 0.5 * hp * c_g16w[j] * sp;
  }
  dW[(size_t)blockIdx.x * (kNearQ * 4) + j * 4 + ab] = acc;
}

// One warp per corrected node: lane l takes entries l and l + 32 of each pair's 64 weights (node j =
// e / 4, component pair e % 4), so a warp reads a pair's 512 bytes in two coalesced loads; the two
// velocity components are reduced across the warp in a fixed order.
__global__ void k_near_apply(long long n_nodes, const long long* node, const long long* ptr, const int* panel,
                             const double* dW, const double* mu, long long N, double* u) {
  const long long k = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= n_nodes) return;
  double s0 = 0.0, s1 = 0.0;
  for (long long p = ptr[k]; p < ptr[k + 1]; ++p) {
    const double* w = dW + p * (kNearQ * 4);
    const long long base = (long long)panel[p] * kNearQ;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = lane + 32 * h, j = e >> 2, c = e & 3;
      const double v = w[e] * mu[2 * (base + j) + (c & 1)];
      if (c < 2) s0 += v; else s1 += v;
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if (lane == 0) {
    const long long o = node[k];
    u[o] += s0;
    u[N + o] += s1;
  }
}

}  // namespace

int launch_near_weights(double alpha, StarGeom g, const NearPair* pairs, long long n_pairs, double* dW,
                        cudaStream_t s) {
  if (n_pairs <= 0) return VP_OK;
  static bool rules = false;
  if (!rules) {
    std::vector<double> x20(kGQ), w20(kGQ), x16(kNearQ), w16(kNearQ), bw(kNearQ);
    gauss_legendre_host(kGQ, x20.data(), w20.data());
    gauss_legendre_host(kNearQ, x16.data(), w16.data());
    for (int i = 0; i < kNearQ; ++i) {
      double prod = 1.0;
      for (int m = 0; m < kNearQ; ++m) if (m != i) prod *= x16[i] - x16[m];
      bw[i] = 1.0 / prod;
    }
    TRY(cudaMemcpyToSymbol(c_g20x, x20.data(), kGQ * sizeof(double)));
    TRY(cudaMemcpyToSymbol(c_g20w, w20.data(), kGQ * sizeof(double)));
    TRY(cudaMemcpyToSymbol(c_g16x, x16.data(), kNearQ * sizeof(double)));
    TRY(cudaMemcpyToSymbol(c_g16w, w16.data(), kNearQ * sizeof(double)));
    TRY(cudaMemcpyToSymbol(c_bw16n, bw.data(), kNearQ * sizeof(double)));
    rules = true;
  }
  for (long long p0 = 0; p0 < n_pairs; p0 += 1 << 30) {
    const long long np = std::min<long long>(n_pairs - p0, 1 << 30);
    k_near_weights<<<(unsigned)np, 64, 0, s>>>(alpha, g, pairs + p0, dW + p0 * kNearQ * 4);
    TRY(cudaGetLastError());
  }
  return VP_OK;
}

int launch_near_apply(long long n_nodes, const long long* node, const long long* ptr, const int* panel,
                      const double* dW, const double* mu, long long N, double* u, cudaStream_t s) {
  if (n_nodes <= 0) return VP_OK;
  k_near_apply<<<(unsigned)((n_nodes * 32 + 255) / 256), 256, 0, s>>>(n_nodes, node, ptr, panel, dW, mu, N, u);
  TRY(cudaGetLastError());
  return VP_OK;
}

}  // namespace vp
