// Boundary integral equation of the homogeneous modified Stokes problem and its GMRES solver.
//
// Sec. 2.2 (Eqs. uH_dbl, dbl_lyr_pot, dbl_lyr_ker, BIE): u^H = D[mu] with the double-layer kernel
// D_ij(x, y) = -T_jik(x - y) n_k(y), n the unit normal pointing into the domain, and the density
// solves 1/2 mu + D[mu] + W[mu] = g on the boundary, W[mu](x) = n(x) / |boundary| * int mu.n ds.
// The stresslet T is the closed form of App. B (Eq. app_stresslet with T1, T2, T3), evaluated by the
// power series of App. C for small alpha r; the stokeslet S (Eq. app_stokeslet) gives exact solutions
// for tests. Discretisation (Sec. 3.2, Eq. BIE_quad): the boundary is a star r(t) = R + A cos(k t + phi),
// split into n_panels equal parameter panels with 16 Gauss-Legendre nodes each (Nystrom). Entries
// for source panels adjacent to (or containing) the target use a locally graded quadrature: the
// panel is cut at the target (self panel) or toward the nearer end (neighbours) into geometrically
// shrinking pieces with 12-point Gauss-Legendre each, the density interpolated by the panel's
// Lagrange basis; this integrates the r log r terms of the kernel (which make plain Gauss-Legendre
// converge slowly, Sec. 4.1) to full precision. The coincident-point limit of the kernel is
// kappa t t / (2 pi) (Sec. 4.2).
// The dense FP64 system (2N x 2N) is solved by GMRES with classical Gram-Schmidt applied twice.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <memory>
#include <new>
#include <vector>

#include "special.cuh"
#include "stokes.cuh"
#include "vp_internal.h"
#include "../../include/bie.h"

namespace vp {
namespace {

#define TRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_last_cuda(e_); return e_ == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA; } } while (0)

constexpr int kPP = 16;        // nodes per panel
constexpr int kGradeN = 12;    // nodes per graded piece
constexpr int kGradeLevels = 36;

__constant__ double c_glx16[kPP], c_glw16[kPP], c_glx12[kGradeN], c_glw12[kGradeN], c_bw16[kPP];

struct Star { double R, A, phase; int k; };

__device__ inline void star_geom(const Star& s, double t, double& x, double& y, double& dx, double& dy,
                                 double& ddx, double& ddy) {
  const double c = cos(t), sn = sin(t);
  const double r = s.R + s.A * cos(s.k * t + s.phase);
  const double dr = -s.A * s.k * sin(s.k * t + s.phase);
  const double d2r = -s.A * s.k * s.k * cos(s.k * t + s.phase);
  x = r * c; y = r * sn;
  dx = dr * c - r * sn; dy = dr * sn + r * c;
  ddx = d2r * c - 2.0 * dr * sn - r * c;
  ddy = d2r * sn + 2.0 * dr * c - r * sn;
}

__device__ inline double lag16(double tau, int j) {
  double num = 0.0, den = 0.0;
  for (int m = 0; m < kPP; ++m) {
    const double d = tau - c_glx16[m];
    if (d == 0.0) return m == j ? 1.0 : 0.0;
    const double w = c_bw16[m] / d;
    den += w;
    if (m == j) num = w;
  }
  return num / den;
}

struct Nodes {
  double *x, *y, *nx, *ny, *w, *kappa, *tx, *ty, *theta;
};

__global__ void k_nodes(Star s, int np, Nodes nd) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= np * kPP) return;
  const int p = j / kPP, q = j % kPP;
  const double h = 2.0 * kPi / np;
  const double t = (p + 0.5) * h + 0.5 * h * c_glx16[q];
  double x, y, dx, dy, ddx, ddy;
  star_geom(s, t, x, y, dx, dy, ddx, ddy);
  const double sp = sqrt(dx * dx + dy * dy);
  nd.x[j] = x; nd.y[j] = y;
  nd.tx[j] = dx / sp; nd.ty[j] = dy / sp;
  nd.nx[j] = -dy / sp; nd.ny[j] = dx / sp;  // counter-clockwise curve: left normal points inside
  nd.w[j] = sp * 0.5 * h * c_glw16[q];
  nd.kappa[j] = (dx * ddy - dy * ddx) / (sp * sp * sp);
  nd.theta[j] = t;
}

// Plain Nystrom entries (row-major [2N][2N]) with the W term and the coincident-point limit.
__global__ void k_matrix_plain(int N, double alpha, double Lb, Nodes nd, double* A) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)N * N) return;
  const int i = (int)(idx / N), j = (int)(idx % N);
  double D[4];
  if (i == j) {
    const double c = nd.kappa[j] / (2.0 * kPi);
    D[0] = c * nd.tx[j] * nd.tx[j]; D[1] = c * nd.tx[j] * nd.ty[j];
    D[2] = D[1]; D[3] = c * nd.ty[j] * nd.ty[j];
  } else {
    dl_kernel(alpha, nd.x[i] - nd.x[j], nd.y[i] - nd.y[j], nd.nx[j], nd.ny[j], D);
  }
  const double w = nd.w[j];
  const double ni[2] = {nd.nx[i], nd.ny[i]}, nj[2] = {nd.nx[j], nd.ny[j]};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      A[(size_t)(2 * i + a) * (2 * N) + 2 * j + b] =
          (i == j && a == b ? 0.5 : 0.0) + D[2 * a + b] * w + ni[a] * nj[b] * w / Lb;
}

// Graded local quadrature: for target i and source panels p-1, p, p+1, the exact (to quadrature
// precision) integral of the kernel against each Lagrange basis function of the source panel.
__global__ void __launch_bounds__(128) k_matrix_local(int np, double alpha, double Lb, Star s, Nodes nd, double* A) {
  const int i = blockIdx.x;
  const int N = np * kPP;
  const int pi = i / kPP;
  const double h = 2.0 * kPi / np;
  const double ti = nd.theta[i];
  const double xi = nd.x[i], yi = nd.y[i];
  // accumulators: 3 panels x 16 basis x 4 components
  __shared__ double acc[3 * kPP * 4];
  for (int e = threadIdx.x; e < 3 * kPP * 4; e += blockDim.x) acc[e] = 0.0;
  __syncthreads();
  // pieces: for each of the 3 panels, 2 sides x (levels + 1) pieces, 12 nodes each
  const int pieces_per_side = kGradeLevels + 1;
  const int npts = 3 * 2 * pieces_per_side * kGradeN;
  for (int e = threadIdx.x; e < npts; e += blockDim.x) {
    const int pn = e / (2 * pieces_per_side * kGradeN);
    int rem = e % (2 * pieces_per_side * kGradeN);
    const int side = rem / (pieces_per_side * kGradeN);
    rem %= pieces_per_side * kGradeN;
    const int lev = rem / kGradeN, q = rem % kGradeN;
    const int p = (pi + pn - 1 + np) % np;
    // panel parameter interval, unwrapped next to the target's panel
    const double ta = (pi + pn - 1) * h, tb = ta + h;
    // grading point: the target (self panel) or the panel end nearest to it (neighbours)
    const double tc = (pn == 1) ? ti : (pn == 0 ? tb : ta);
    const double lo_end = side == 0 ? ta : tc, hi_end = side == 0 ? tc : tb;
    const double len = hi_end - lo_end;
    if (len <= 0.0) continue;
    // geometric pieces toward tc: side 0 grades toward hi_end = tc, side 1 toward lo_end = tc
    double u0, u1;  // fractions of len measured from tc
    if (lev == kGradeLevels) { u0 = 0.0; u1 = ldexp(1.0, -kGradeLevels); }
    else { u0 = ldexp(1.0, -lev - 1); u1 = ldexp(1.0, -lev); }
    const double fa = 0.5 * (u0 + u1) + 0.5 * (u1 - u0) * c_glx12[q];
    const double wq = 0.5 * (u1 - u0) * c_glw12[q] * len;
    const double t = (side == 0) ? (tc - fa * len) : (tc + fa * len);
    if (!(t > ta && t < tb) && !(t == ta || t == tb)) continue;
    double x, y, dx, dy, ddx, ddy;
    star_geom(s, t, x, y, dx, dy, ddx, ddy);
    const double sp = sqrt(dx * dx + dy * dy);
    const double nxq = -dy / sp, nyq = dx / sp;
    // x_i - y(t) from the parameter offset, free of cancellation:
    // z(ti) - z(t) = e^{i ti} [ (r(ti) - r(t)) + r(t) (1 - e^{i d}) ],  d = t - ti,
    // r(ti) - r(t) = 2 A sin(k (ti + t)/2 + phase) sin(k d / 2),  1 - e^{i d} = 2 sin^2(d/2) - i sin d
    const double d = (tc - ti) + ((side == 0) ? -fa * len : fa * len);
    const double rt = s.R + s.A * cos(s.k * t + s.phase);
    const double dR = 2.0 * s.A * sin(0.5 * s.k * (ti + t) + s.phase) * sin(0.5 * s.k * d);
    const double sh = sin(0.5 * d);
    const double re = dR + rt * 2.0 * sh * sh, im = -rt * sin(d);
    const double ct = cos(ti), st = sin(ti);
    const double rx = ct * re - st * im, ry = st * re + ct * im;
    if (rx == 0.0 && ry == 0.0) continue;
    (void)x; (void)y; (void)xi; (void)yi;
    double D[4];
    dl_kernel(alpha, rx, ry, nxq, nyq, D);
    const double tau = 2.0 * (t - ta) / h - 1.0;  // reference coordinate on the source panel
    for (int j = 0; j < kPP; ++j) {
      const double l = lag16(tau, j) * wq * sp;
      for (int c = 0; c < 4; ++c) atomicAdd(&acc[(pn * kPP + j) * 4 + c], D[c] * l);
    }
    (void)p;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 3 * kPP; e += blockDim.x) {
    const int pn = e / kPP, jj = e % kPP;
    const int p = (pi + pn - 1 + np) % np;
    const int j = p * kPP + jj;
    const double ni[2] = {nd.nx[i], nd.ny[i]}, nj[2] = {nd.nx[j], nd.ny[j]};
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        A[(size_t)(2 * i + a) * (2 * N) + 2 * j + b] =
            (i == j && a == b ? 0.5 : 0.0) + acc[(pn * kPP + jj) * 4 + 2 * a + b] + ni[a] * nj[b] * nd.w[j] / Lb;
  }
}

// y = A x for a dense row-major n x n FP64 matrix: one warp per row.
// GMRES state on the device; every Krylov kernel returns at once when `done` is set, so the host
// can queue several iterations ahead and look at the state only once per group.
struct GmresCtl {
  double bnorm, res, hn;
  int done, it;
};

__device__ inline bool gm_done(const GmresCtl* c) { return c && *(volatile const int*)&c->done; }

// y = A x, A row-major n x n (n even): one warp per row. The matrix is streamed once
// (loads that bypass L1, four 16-byte loads in flight per lane); x stays in L1/L2.
__global__ void k_gemv(int n, const double* __restrict__ A, const double* __restrict__ x, double* __restrict__ y,
                       const GmresCtl* ctl = nullptr) {
  if (gm_done(ctl)) return;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double2* a = reinterpret_cast<const double2*>(A + (size_t)row * n);
  const double2* xv = reinterpret_cast<const double2*>(x);
  const int n2 = n >> 1;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int k = lane;
  for (; k + 96 < n2; k += 128) {
    const double2 a0 = __ldcs(a + k), a1 = __ldcs(a + k + 32), a2 = __ldcs(a + k + 64), a3 = __ldcs(a + k + 96);
    const double2 x0 = __ldg(xv + k), x1 = __ldg(xv + k + 32), x2 = __ldg(xv + k + 64), x3 = __ldg(xv + k + 96);
    s0 = fma(a0.x, x0.x, fma(a0.y, x0.y, s0));
    s1 = fma(a1.x, x1.x, fma(a1.y, x1.y, s1));
    s2 = fma(a2.x, x2.x, fma(a2.y, x2.y, s2));
    s3 = fma(a3.x, x3.x, fma(a3.y, x3.y, s3));
  }
  for (; k < n2; k += 32) {
    const double2 a0 = __ldcs(a + k), x0 = __ldg(xv + k);
    s0 = fma(a0.x, x0.x, fma(a0.y, x0.y, s0));
  }
  double s = (s0 + s1) + (s2 + s3);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = s;
}

// h[c] = sum_k V[c][k] w[k] for c < ncols (V row-major [ncols][n]): one block per column.
__global__ void k_dots(int n, int ncols, const double* __restrict__ V, const double* __restrict__ w, double* h,
                       const GmresCtl* ctl = nullptr) {
  if (gm_done(ctl)) return;
  const int c = blockIdx.x;
  if (c >= ncols) return;
  __shared__ double red[32];
  double s = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) s += V[(size_t)c * n + k] * w[k];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) h[c] = s;
  }
}

// w -= sum_c h[c] V[c]
__global__ void k_sub_proj(int n, int ncols, const double* __restrict__ V, const double* __restrict__ h, double* w,
                           const GmresCtl* ctl = nullptr) {
  if (gm_done(ctl)) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s = w[k];
  for (int c = 0; c < ncols; ++c) s -= h[c] * V[(size_t)c * n + k];
  w[k] = s;
}

__global__ void k_axpby(int n, double a, const double* x, double b, double* y) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) y[k] = a * x[k] + b * y[k];
}

// x += sum_{c < it} y[c] V[c], it the iteration count in the GMRES state
__global__ void k_add_comb(int n, const GmresCtl* ctl, const double* __restrict__ V, const double* __restrict__ coef,
                           double* x) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int ncols = ctl->it;
  double s = x[k];
  for (int c = 0; c < ncols; ++c) s += coef[c] * V[(size_t)c * n + k];
  x[k] = s;
}

// Start of GMRES (one thread): norms from the dot products gr = (g.g, r.r).
__global__ void k_gm_init(GmresCtl* ctl, const double* gr, double tol, double* gv) {
  const double bnorm = gr[0] > 0.0 ? sqrt(gr[0]) : 1.0, beta = sqrt(fmax(gr[1], 0.0));
  ctl->bnorm = bnorm;
  ctl->res = beta / bnorm;
  ctl->hn = beta;
  ctl->it = 0;
  ctl->done = (beta / bnorm <= tol || beta == 0.0) ? 1 : 0;
  gv[0] = beta;
}

// y = x / ctl->hn (the next Krylov vector), skipped once converged.
__global__ void k_gm_scale(int n, const GmresCtl* ctl, const double* __restrict__ x, double* __restrict__ y) {
  if (gm_done(ctl)) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) y[k] = x[k] / ctl->hn;
}

// Arnoldi step j (one thread): Hessenberg column j from the two Gram-Schmidt passes hv0, hv1 and
// |w|^2, earlier Givens rotations applied, new rotation, residual estimate |gv[j+1]| / |g|.
__global__ void k_gm_step(int j, int m, double tol, GmresCtl* ctl, double* H, double* cs, double* sn, double* gv,
                          const double* hv0, const double* hv1, const double* wn2) {
  if (ctl->done) return;
  for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hv0[i] + hv1[i];
  const double hn = sqrt(fmax(*wn2, 0.0));
  H[(size_t)(j + 1) * m + j] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
    H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
    H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
  }
  const double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
  const double d = hypot(a, c);
  cs[j] = d > 0.0 ? a / d : 1.0;
  sn[j] = d > 0.0 ? c / d : 0.0;
  H[(size_t)j * m + j] = d;
  H[(size_t)(j + 1) * m + j] = 0.0;
  gv[j + 1] = -sn[j] * gv[j];
  gv[j] = cs[j] * gv[j];
  ctl->it = j + 1;
  ctl->hn = hn;
  ctl->res = fabs(gv[j + 1]) / ctl->bnorm;
  if (ctl->res <= tol || hn == 0.0) ctl->done = 1;
}

// Augmentation by a direction d (w = A d on entry): with s = (w.r)/(w.w), mu += s d, r -= s w
// (the least-squares step along d), c = w/|w|, u = d/|w|; nothing when w = 0.
__global__ void k_aug_setup(int n, const double* ww_wr, const double* w, const double* d, double* r, double* mu,
                            double* c, double* u) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double ww = ww_wr[0], wr = ww_wr[1];
  if (!(ww > 0.0)) {
    c[k] = 0.0;
    u[k] = 0.0;
    return;
  }
  const double nrm = sqrt(ww), st = wr / ww;
  mu[k] += st * d[k];
  r[k] -= st * w[k];
  c[k] = w[k] / nrm;
  u[k] = d[k] / nrm;
}

// w -= beta c, beta = *bj (the component of A v_j along c, removed from the Krylov operator).
__global__ void k_aug_project(int n, const GmresCtl* ctl, const double* bj, const double* c, double* w) {
  if (gm_done(ctl)) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) w[k] -= *bj * c[k];
}

// mu -= (sum_{j < it} b_j y_j) u: the update V y moved A mu by the removed components c b.y.
__global__ void k_aug_final(int n, const GmresCtl* ctl, const double* bv, const double* y, const double* u,
                            double* mu) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double sdot = 0.0;
  for (int j = 0; j < ctl->it; ++j) sdot += bv[j] * y[j];
  mu[k] -= sdot * u[k];
}

// Least-squares solution of the rotated Hessenberg system (one thread, back substitution).
__global__ void k_gm_backsub(int m, const GmresCtl* ctl, const double* H, const double* gv, double* y) {
  const int it = ctl->it;
  for (int i = it - 1; i >= 0; --i) {
    double t = gv[i];
    for (int k = i + 1; k < it; ++k) t -= H[(size_t)i * m + k] * y[k];
    y[i] = t / H[(size_t)i * m + i];
  }
}

// u(x_t) = sum_j D(x_t, y_j) mu_j w_j (targets away from the boundary).
__global__ void k_eval_dl(int N, double alpha, Nodes nd, const double* mu, int M, const double* txy, double* u) {
  const int t = blockIdx.x;
  if (t >= M) return;
  const double x = txy[t], y = txy[M + t];
  double s0 = 0.0, s1 = 0.0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    double D[4];
    dl_kernel(alpha, x - nd.x[j], y - nd.y[j], nd.nx[j], nd.ny[j], D);
    const double w = nd.w[j];
    s0 += (D[0] * mu[2 * j] + D[1] * mu[2 * j + 1]) * w;
    s1 += (D[2] * mu[2 * j] + D[3] * mu[2 * j + 1]) * w;
  }
  __shared__ double r0[256], r1[256];
  r0[threadIdx.x] = s0; r1[threadIdx.x] = s1;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if ((int)threadIdx.x < o) { r0[threadIdx.x] += r0[threadIdx.x + o]; r1[threadIdx.x] += r1[threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { u[t] = r0[0]; u[M + t] = r1[0]; }
}

// Stokeslet sum at points: u_a(x) = sum_k S_ab(x - s_k) f_kb.
__global__ void k_stokeslets(double alpha, int K, const double* src, const double* f, int M, const double* xy,
                             double* u) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= M) return;
  double u0 = 0.0, u1 = 0.0;
  for (int k = 0; k < K; ++k) {
    const double rx = xy[t] - src[2 * k], ry = xy[M + t] - src[2 * k + 1];
    const double r = sqrt(rx * rx + ry * ry);
    double T1, T2, T3, S1, S2;
    stress_funcs(alpha * r, T1, T2, T3, S1, S2);
    const double a2 = alpha * alpha;
    u0 += (S1 + a2 * S2 * rx * rx) * f[2 * k] + a2 * S2 * rx * ry * f[2 * k + 1];
    u1 += a2 * S2 * rx * ry * f[2 * k] + (S1 + a2 * S2 * ry * ry) * f[2 * k + 1];
  }
  u[t] = u0;
  u[M + t] = u1;
}

// Kernel scalars at given z (for tests): out[5][n] = T1, T2, T3, S1, S2.
__global__ void k_stress_funcs(int n, const double* z, double* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double T1, T2, T3, S1, S2;
  stress_funcs(z[t], T1, T2, T3, S1, S2);
  out[t] = T1; out[n + t] = T2; out[2 * n + t] = T3; out[3 * n + t] = S1; out[4 * n + t] = S2;
}

void gl_host(int n, double* x, double* w) { gauss_legendre_host(n, x, w); }

}  // namespace
}  // namespace vp

struct bie_s {
  int np = 0, N = 0, n2 = 0;
  double alpha = 0.0, Lb = 0.0;
  vp::Star star{};
  vp::Nodes nd{};
  std::vector<void*> allocs;
  double* A = nullptr;
  // GMRES work space
  int m = 0;
  double *V = nullptr, *w = nullptr, *r = nullptr;
  double* gm = nullptr;          // H [(m+1) m], cs [m], sn [m], gv [m+2], y [m], hv [2(m+1)], scalars [8]
  double *ac = nullptr, *au = nullptr, *abv = nullptr;  // augmentation: c, u [2N], b [m]
  vp::GmresCtl* ctl = nullptr;   // device
  vp::GmresCtl* hctl = nullptr;  // pinned host copy
};

using namespace vp;

namespace {
template <class T>
int dalloc(bie_s* b, T** p, size_t n) {
  void* q = nullptr;
  TRY(cudaMalloc(&q, std::max<size_t>(1, n) * sizeof(T)));
  b->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return VP_OK;
}
}  // namespace

extern "C" void bie_free(bie b) {
  if (!b) return;
  if (b->hctl) cudaFreeHost(b->hctl);
  for (void* p : b->allocs) cudaFree(p);
  delete b;
}

extern "C" int bie_create(double alpha, double R, double A, int k, double phase, int n_panels, int max_krylov,
                          void* stream, bie* out) {
  if (!out) return VP_ERR_ARG;
  *out = nullptr;
  if (!(alpha > 0.0) || !(R > 0.0) || !(A >= 0.0) || A >= R || k < 0 || n_panels < 4 || n_panels > 4096 ||
      max_krylov < 1 || max_krylov > 1000)
    return VP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::unique_ptr<bie_s> B(new (std::nothrow) bie_s());
  if (!B) return VP_ERR_OOM;
  B->np = n_panels; B->N = n_panels * kPP; B->n2 = 2 * B->N; B->alpha = alpha;
  B->star = {R, A, phase, k};
  B->m = max_krylov;
  {
    double x16[kPP], w16[kPP], x12[kGradeN], w12[kGradeN], bw[kPP];
    gl_host(kPP, x16, w16);
    gl_host(kGradeN, x12, w12);
    for (int i = 0; i < kPP; ++i) {
      double prod = 1.0;
      for (int j = 0; j < kPP; ++j) if (j != i) prod *= x16[i] - x16[j];
      bw[i] = 1.0 / prod;
    }
    TRY(cudaMemcpyToSymbolAsync(c_glx16, x16, sizeof(x16), 0, cudaMemcpyHostToDevice, s));
    TRY(cudaMemcpyToSymbolAsync(c_glw16, w16, sizeof(w16), 0, cudaMemcpyHostToDevice, s));
    TRY(cudaMemcpyToSymbolAsync(c_glx12, x12, sizeof(x12), 0, cudaMemcpyHostToDevice, s));
    TRY(cudaMemcpyToSymbolAsync(c_glw12, w12, sizeof(w12), 0, cudaMemcpyHostToDevice, s));
    TRY(cudaMemcpyToSymbolAsync(c_bw16, bw, sizeof(bw), 0, cudaMemcpyHostToDevice, s));
  }
  int rc;
  const int N = B->N;
  Nodes& nd = B->nd;
  for (double** p : {&nd.x, &nd.y, &nd.nx, &nd.ny, &nd.w, &nd.kappa, &nd.tx, &nd.ty, &nd.theta})
    if ((rc = dalloc(B.get(), p, N))) { bie_free(B.release()); return rc; }
  if ((rc = dalloc(B.get(), &B->A, (size_t)B->n2 * B->n2))) { bie_free(B.release()); return rc; }
  if ((rc = dalloc(B.get(), &B->V, (size_t)(B->m + 1) * B->n2)) || (rc = dalloc(B.get(), &B->w, B->n2)) ||
      (rc = dalloc(B.get(), &B->r, B->n2)) ||
      (rc = dalloc(B.get(), &B->gm, (size_t)(B->m + 1) * B->m + 6 * (size_t)B->m + 12)) ||
      (rc = dalloc(B.get(), &B->ctl, 1)) || (rc = dalloc(B.get(), &B->ac, B->n2)) ||
      (rc = dalloc(B.get(), &B->au, B->n2)) || (rc = dalloc(B.get(), &B->abv, B->m))) {
    bie_free(B.release());
    return rc;
  }
  if (cudaHostAlloc(&B->hctl, sizeof(GmresCtl), cudaHostAllocDefault) != cudaSuccess) {
    B->hctl = nullptr;
    bie_free(B.release());
    return VP_ERR_OOM;
  }
  k_nodes<<<(N + 127) / 128, 128, 0, s>>>(B->star, B->np, nd);
  // boundary length
  std::vector<double> w(N);
  if (cudaMemcpyAsync(w.data(), nd.w, N * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    bie_free(B.release());
    return VP_ERR_CUDA;
  }
  double L = 0.0;
  for (double v : w) L += v;
  B->Lb = L;
  const long long NN = (long long)N * N;
  k_matrix_plain<<<(unsigned)((NN + 255) / 256), 256, 0, s>>>(N, alpha, L, nd, B->A);
  k_matrix_local<<<N, 128, 0, s>>>(B->np, alpha, L, B->star, nd, B->A);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    bie_free(B.release());
    return VP_ERR_CUDA;
  }
  *out = B.release();
  return VP_OK;
}

extern "C" int bie_size(bie b, int* n_nodes, double* boundary_length) {
  if (!b) return VP_ERR_ARG;
  if (n_nodes) *n_nodes = b->N;
  if (boundary_length) *boundary_length = b->Lb;
  return VP_OK;
}

extern "C" int bie_nodes(bie b, double* out, void* stream) {
  if (!b || !out) return VP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int N = b->N;
  const double* src[7] = {b->nd.x, b->nd.y, b->nd.nx, b->nd.ny, b->nd.w, b->nd.kappa, b->nd.theta};
  for (int k = 0; k < 7; ++k)
    TRY(cudaMemcpyAsync(out + (size_t)k * N, src[k], N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return VP_OK;
}

extern "C" int bie_apply(bie b, const double* mu, double* out, void* stream) {
  if (!b || !mu || !out || (reinterpret_cast<uintptr_t>(mu) & 15)) return VP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_gemv<<<(b->n2 * 32 + 255) / 256, 256, 0, s>>>(b->n2, b->A, mu, out);
  TRY(cudaGetLastError());
  return VP_OK;
}

extern "C" int bie_solve_aug(bie b, const double* g, double* mu, const double* d, double tol, int max_iter,
                             int* iters, double* relres, void* stream) {
  if (!b || !g || !mu || !(tol > 0.0) || max_iter < 1 || (reinterpret_cast<uintptr_t>(mu) & 15) ||
      (reinterpret_cast<uintptr_t>(d) & 15))
    return VP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n = b->n2, M = b->m;
  const int m = std::min(max_iter, M);
  const int T = 256, G = (n + T - 1) / T, GV = (n * 32 + 255) / 256;
  double* H = b->gm;
  double* cs = H + (size_t)(M + 1) * M;
  double* sn = cs + M;
  double* gv = sn + M;
  double* y = gv + M + 2;
  double* hv = y + M;
  double* wn2 = hv + 2 * (M + 1);
  GmresCtl* ctl = b->ctl;
  // r = g - A mu, norms, V0 = r / |r|
  k_gemv<<<GV, 256, 0, s>>>(n, b->A, mu, b->r);
  k_axpby<<<G, T, 0, s>>>(n, 1.0, g, -1.0, b->r);
  if (d) {
    // least-squares step along d, then GMRES on (I - c c^T) A so that direction stays removed
    k_gemv<<<GV, 256, 0, s>>>(n, b->A, d, b->w);
    k_dots<<<1, 256, 0, s>>>(n, 1, b->w, b->w, wn2 + 4);
    k_dots<<<1, 256, 0, s>>>(n, 1, b->w, b->r, wn2 + 5);
    k_aug_setup<<<G, T, 0, s>>>(n, wn2 + 4, b->w, d, b->r, mu, b->ac, b->au);
  }
  k_dots<<<1, 256, 0, s>>>(n, 1, g, g, wn2);
  k_dots<<<1, 256, 0, s>>>(n, 1, b->r, b->r, wn2 + 1);
  k_gm_init<<<1, 1, 0, s>>>(ctl, wn2, tol, gv);
  k_gm_scale<<<G, T, 0, s>>>(n, ctl, b->r, b->V);
  // Arnoldi with classical Gram-Schmidt applied twice; the host queues kGroup iterations at a time
  // and reads the device state after each group (iterations past convergence are no-ops).
  constexpr int kGroup = 4;
  for (int j = 0; j < m;) {
    const int jend = std::min(m, j + kGroup);
    for (; j < jend; ++j) {
      const double* vj = b->V + (size_t)j * n;
      k_gemv<<<GV, 256, 0, s>>>(n, b->A, vj, b->w, ctl);
      if (d) {
        k_dots<<<1, 256, 0, s>>>(n, 1, b->ac, b->w, b->abv + j, ctl);
        k_aug_project<<<G, T, 0, s>>>(n, ctl, b->abv + j, b->ac, b->w);
      }
      for (int pass = 0; pass < 2; ++pass) {
        k_dots<<<j + 1, 256, 0, s>>>(n, j + 1, b->V, b->w, hv + pass * (M + 1), ctl);
        k_sub_proj<<<G, T, 0, s>>>(n, j + 1, b->V, hv + pass * (M + 1), b->w, ctl);
      }
      k_dots<<<1, 256, 0, s>>>(n, 1, b->w, b->w, wn2 + 2, ctl);
      k_gm_step<<<1, 1, 0, s>>>(j, M, tol, ctl, H, cs, sn, gv, hv, hv + M + 1, wn2 + 2);
      k_gm_scale<<<G, T, 0, s>>>(n, ctl, b->w, b->V + (size_t)(j + 1) * n);
    }
    TRY(cudaMemcpyAsync(b->hctl, ctl, sizeof(GmresCtl), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    if (b->hctl->done) break;
  }
  // update and the true residual
  k_gm_backsub<<<1, 1, 0, s>>>(M, ctl, H, gv, y);
  k_add_comb<<<G, T, 0, s>>>(n, ctl, b->V, y, mu);
  if (d) k_aug_final<<<G, T, 0, s>>>(n, ctl, b->abv, y, b->au, mu);
  k_gemv<<<GV, 256, 0, s>>>(n, b->A, mu, b->r);
  k_axpby<<<G, T, 0, s>>>(n, 1.0, g, -1.0, b->r);
  k_dots<<<1, 256, 0, s>>>(n, 1, b->r, b->r, wn2 + 3);
  double rr[2] = {0.0, 0.0};
  TRY(cudaMemcpyAsync(b->hctl, ctl, sizeof(GmresCtl), cudaMemcpyDeviceToHost, s));
  TRY(cudaMemcpyAsync(rr, wn2 + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  if (iters) *iters = b->hctl->it;
  if (relres) *relres = std::sqrt(std::max(rr[0], 0.0)) / b->hctl->bnorm;
  TRY(cudaGetLastError());
  return VP_OK;
}

extern "C" int bie_solve(bie b, const double* g, double* mu, double tol, int max_iter, int* iters, double* relres,
                         void* stream) {
  return bie_solve_aug(b, g, mu, nullptr, tol, max_iter, iters, relres, stream);
}

extern "C" int bie_eval(bie b, const double* mu, int n_targets, const double* txy, double* u, void* stream) {
  if (!b || !mu || !txy || !u || n_targets < 0) return VP_ERR_ARG;
  if (n_targets == 0) return VP_OK;
  k_eval_dl<<<n_targets, 256, 0, static_cast<cudaStream_t>(stream)>>>(b->N, b->alpha, b->nd, mu, n_targets, txy, u);
  TRY(cudaGetLastError());
  return VP_OK;
}

extern "C" int bie_stokeslets(double alpha, int n_sources, const double* src, const double* f, int n_points,
                              const double* xy, double* u, void* stream) {
  if (!(alpha > 0.0) || n_sources < 0 || n_points < 0 || !src || !f || !xy || !u) return VP_ERR_ARG;
  if (n_points == 0) return VP_OK;
  k_stokeslets<<<(n_points + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(alpha, n_sources, src, f,
                                                                                       n_points, xy, u);
  TRY(cudaGetLastError());
  return VP_OK;
}

extern "C" int bie_kernel_scalars(int n, const double* z, double* out, void* stream) {
  if (n < 0 || !z || !out) return VP_ERR_ARG;
  if (n == 0) return VP_OK;
  k_stress_funcs<<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(n, z, out);
  TRY(cudaGetLastError());
  return VP_OK;
}
