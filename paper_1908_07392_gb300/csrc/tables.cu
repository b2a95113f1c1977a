// Table and operator builder: vp_tables_build / vp_tables_free.
//
// Everything is built on the device in FP64 for levels 0..L of a root box of
// side `side` (leaf side h_l = side / 2^l).
//
// Near tables (Sec. 2.1, Eq. vol_pot, restricted to adjacent leaves): for a
// target leaf [0,h]^2 and a source leaf at one of the 33 adjacent relative
// positions, entry [f*n + t][k] is the integral over the source leaf of
// (G, dG/dx, dG/dy)(x_t - y) times the Lagrange basis function k of the source
// leaf.  Quadrature: the source leaf is subdivided toward x_t until every piece
// lies at least 0.75 of its longest side away (then tensor Gauss-Legendre of
// order 20, or 16 beyond two sides); for the self position the square centred
// at x_t that touches the nearest leaf edge is integrated in polar coordinates
// (four right isosceles triangles, 20-point Gauss-Legendre in angle, radial
// panels [R 2^-(k+1), R 2^-k] with 12-point Gauss-Legendre each), which absorbs
// the log r and 1/r singularities of G and grad G.
//
// Expansion operators (Sec. 3.2.1, Eqs. mpole and loc, with the K_n / I_n part
// and, for the modified-biharmonic kernel, the log / r^|n| part as separate
// channels; real cos/sin modes; every basis function is normalised to be
// cos(m theta) or sin(m theta) on the circumcircle of its box):
//  S2M   analytic moments: from the addition theorem
//        K0(a|x-y|) = sum_m K_m(a rho_x) I_m(a rho_y) cos(m(theta_x - theta_y))
//        and log|x-y| = log rho_x - sum_{m>=1} (rho_y/rho_x)^m cos(m(...))/m,
//        integrated against the Lagrange basis with tensor Gauss-Legendre of order 40
//        (exact for the polynomial part), on more sub-boxes when alpha h is large.
//  M2M, M2L, L2L   the target coefficients are the Fourier coefficients of the
//        source basis function sampled at Q points on the target box's circle;
//        the constant mode of a log multipole is its total charge (carried over
//        exactly by M2M).
//  S2L   Fourier coefficients on the target circle of the source leaf's potential
//        (tensor Gauss-Legendre over the coarse source leaf).
//  L2T, M2T   the basis functions and their gradients evaluated at the nodes.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include "special.cuh"
#include "split.h"
#include "vp_internal.h"

namespace vp {

namespace {
thread_local cudaError_t g_last_cuda = cudaSuccess;
}
void set_last_cuda(cudaError_t e) { g_last_cuda = e; }
cudaError_t last_cuda() { return g_last_cuda; }

const Positions& positions() {
  static const Positions P = [] {
    Positions q;
    std::memset(&q, 0, sizeof(q));
    for (auto* a : {&q.near_same[0][0]}) for (int i = 0; i < 9; ++i) a[i] = -1;
    for (int i = 0; i < 16; ++i) { (&q.near_coarse[0][0])[i] = -1; (&q.near_fine[0][0])[i] = -1; }
    for (int i = 0; i < 36; ++i) { (&q.w_idx[0][0])[i] = -1; (&q.x_idx[0][0])[i] = -1; }
    for (int i = 0; i < 49; ++i) (&q.v_idx[0][0])[i] = -1;
    int k = 0;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) { q.near_same[dy + 1][dx + 1] = k; q.near[k++] = {(double)dx, (double)dy, 1.0}; }
    for (int Y = -2; Y <= 1; ++Y)
      for (int X = -2; X <= 1; ++X) {
        if ((X == -1 || X == 0) && (Y == -1 || Y == 0)) continue;
        q.near_coarse[Y + 2][X + 2] = k; q.near[k++] = {(double)X, (double)Y, 2.0};
      }
    for (int Y = -1; Y <= 2; ++Y)
      for (int X = -1; X <= 2; ++X) {
        if ((X == 0 || X == 1) && (Y == 0 || Y == 1)) continue;
        q.near_fine[Y + 1][X + 1] = k; q.near[k++] = {0.5 * X, 0.5 * Y, 0.5};
      }
    int kw = 0;
    for (int Y = -2; Y <= 3; ++Y)
      for (int X = -2; X <= 3; ++X) {
        if (X >= -1 && X <= 2 && Y >= -1 && Y <= 2) continue;
        q.w_idx[Y + 2][X + 2] = kw; q.w[kw++] = {0.5 * X, 0.5 * Y, 0.5};
      }
    int kx = 0;
    for (int Y = -3; Y <= 2; ++Y)
      for (int X = -3; X <= 2; ++X) {
        const int px = (X & 1) ? -1 : 0, py = (Y & 1) ? -1 : 0;
        const int ax = X - px, ay = Y - py;
        if (!(ax == -2 || ax == 0 || ax == 2) || !(ay == -2 || ay == 0 || ay == 2)) continue;
        if (ax == 0 && ay == 0) continue;
        const bool touch = X <= 1 && X + 2 >= 0 && Y <= 1 && Y + 2 >= 0;
        if (touch) continue;
        q.x_idx[Y + 3][X + 3] = kx; q.x[kx++] = {(double)X, (double)Y, 2.0};
      }
    int kv = 0;
    for (int dy = -3; dy <= 3; ++dy)
      for (int dx = -3; dx <= 3; ++dx) {
        if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
        q.v_idx[dy + 3][dx + 3] = kv; q.v_dx[kv] = dx; q.v_dy[kv] = dy; ++kv;
      }
    if (k != kNearPos || kw != kWPos || kx != kXPos || kv != kVOff) {
      std::fprintf(stderr, "vp: position enumeration mismatch %d %d %d %d\n", k, kw, kx, kv);
    }
    return q;
  }();
  return P;
}

namespace {

constexpr int kMaxQ = 40;
__constant__ double c_gx[kMaxQ + 1][kMaxQ];   // Gauss-Legendre nodes by order
__constant__ double c_gw[kMaxQ + 1][kMaxQ];   // weights
__constant__ double c_bw[16];                  // barycentric weights of the p interpolation nodes

// Gauss-Legendre on [-1,1] (Newton on the Legendre three-term recurrence), ascending.
void host_gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double t = std::cos(kPi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double a = 1.0, b = t;
      for (int k = 2; k <= n; ++k) { double c = ((2.0 * k - 1.0) * t * b - (k - 1.0) * a) / k; a = b; b = c; }
      if (n == 1) { a = 1.0; b = t; }
      const double d = n * (t * b - a) / (t * t - 1.0);
      const double s = b / d;
      t -= s;
      if (std::fabs(s) < 1e-17) break;
    }
    double a = 1.0, b = t;
    for (int k = 2; k <= n; ++k) { double c = ((2.0 * k - 1.0) * t * b - (k - 1.0) * a) / k; a = b; b = c; }
    if (n == 1) { a = 1.0; b = t; }
    const double d = n * (t * b - a) / (t * t - 1.0);
    x[n - 1 - i] = t;
    w[n - 1 - i] = 2.0 / ((1.0 - t * t) * d * d);
  }
}

// Lagrange basis function i of the p-node Gauss-Legendre interpolant at tau (barycentric form).
__device__ inline double lagrange_i(int p, double tau, int i) {
  double num = 0.0, den = 0.0;
  for (int m = 0; m < p; ++m) {
    const double d = tau - c_gx[p][m];
    if (d == 0.0) return (m == i) ? 1.0 : 0.0;
    const double w = c_bw[m] / d;
    den += w;
    if (m == i) num = w;
  }
  return num / den;
}

// ---------------------------------------------------------------- near tables

constexpr int kNT = 256;
constexpr int kMaxRect = 256;
constexpr int kStack = 64;
constexpr int kChunk = 64;
constexpr int kNAng = 20, kNRadPanels = 24, kNRad = 12;

struct Rect { double a1, b1, a2, b2; };

__device__ inline double rect_dist(const Rect& R, double x, double y) {
  const double dx = fmax(fmax(R.a1 - x, 0.0), x - R.b1);
  const double dy = fmax(fmax(R.a2 - y, 0.0), y - R.b2);
  return sqrt(dx * dx + dy * dy);
}

__global__ void __launch_bounds__(kNT) k_near_table(int kernel, double alpha, int p, double h, int self_pos,
                                                    const RelBox* __restrict__ geo, double* __restrict__ out,
                                                    int* __restrict__ err) {
  const int n = p * p;
  const int t = blockIdx.x;
  const int pos = blockIdx.y;
  const RelBox rb = geo[pos];
  const double x = 0.5 * h * (1.0 + c_gx[p][t % p]);
  const double y = 0.5 * h * (1.0 + c_gx[p][t / p]);
  const double sx0 = rb.ox * h, sy0 = rb.oy * h, ss = rb.s * h;

  __shared__ Rect rects[kMaxRect];
  __shared__ int rq[kMaxRect];
  __shared__ int nrect;
  __shared__ double sdel;
  __shared__ double px[24], py[24], wx[24], wy[24];
  __shared__ double Lx[24 * 16], Ly[24 * 16];
  __shared__ double WG[3][kChunk];
  __shared__ Rect stack[kStack];
  // the tensor-rule work arrays and the polar chunk arrays are used in separate phases
  __shared__ double work[3 * 24 * 24 + 3 * 24 * 16];
  double (*G)[24 * 24] = reinterpret_cast<double (*)[24 * 24]>(work);
  double (*H)[24 * 16] = reinterpret_cast<double (*)[24 * 16]>(work + 3 * 24 * 24);
  double* L1 = work;
  double* L2 = work + kChunk * 16;

  if (threadIdx.x == 0) {
    int sp = 0;
    int nr = 0;
    double del = 0.0;
    bool bad = false;
    if (pos == self_pos) {
      del = fmin(fmin(x, h - x), fmin(y, h - y));
      const Rect cand[4] = {{0.0, x - del, 0.0, h}, {x + del, h, 0.0, h}, {x - del, x + del, 0.0, y - del},
                            {x - del, x + del, y + del, h}};
      for (int c = 0; c < 4; ++c)
        if (cand[c].b1 - cand[c].a1 > 0.0 && cand[c].b2 - cand[c].a2 > 0.0) stack[sp++] = cand[c];
    } else {
      stack[sp++] = {sx0, sx0 + ss, sy0, sy0 + ss};
    }
    while (sp > 0 && !bad) {
      const Rect R = stack[--sp];
      const double w = R.b1 - R.a1, hh = R.b2 - R.a2;
      const double s = fmax(w, hh);
      const double d = rect_dist(R, x, y);
      if (d >= 0.75 * s) {
        if (nr >= kMaxRect) { bad = true; break; }
        rects[nr] = R; rq[nr] = (d >= 2.0 * s) ? 16 : 20; ++nr;
        continue;
      }
      if (!(d > 0.0) || sp + 4 > kStack) { bad = true; break; }
      if (w > 2.0 * hh) {
        const double m = 0.5 * (R.a1 + R.b1);
        stack[sp++] = {R.a1, m, R.a2, R.b2}; stack[sp++] = {m, R.b1, R.a2, R.b2};
      } else if (hh > 2.0 * w) {
        const double m = 0.5 * (R.a2 + R.b2);
        stack[sp++] = {R.a1, R.b1, R.a2, m}; stack[sp++] = {R.a1, R.b1, m, R.b2};
      } else {
        const double m1 = 0.5 * (R.a1 + R.b1), m2 = 0.5 * (R.a2 + R.b2);
        stack[sp++] = {R.a1, m1, R.a2, m2}; stack[sp++] = {m1, R.b1, R.a2, m2};
        stack[sp++] = {R.a1, m1, m2, R.b2}; stack[sp++] = {m1, R.b1, m2, R.b2};
      }
    }
    if (bad) { atomicOr(err, 1); nr = 0; del = 0.0; }
    nrect = nr;
    sdel = del;
  }
  __syncthreads();

  const int k = threadIdx.x;
  const int ki = k % p, kj = k / p;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  const double lx0 = (pos == self_pos) ? 0.0 : sx0;  // lower-left of the source leaf
  const double ly0 = (pos == self_pos) ? 0.0 : sy0;
  const double lh = (pos == self_pos) ? h : ss;

  for (int r = 0; r < nrect; ++r) {
    const Rect R = rects[r];
    const int q = rq[r];
    for (int i = threadIdx.x; i < q; i += kNT) {
      px[i] = 0.5 * (R.a1 + R.b1) + 0.5 * (R.b1 - R.a1) * c_gx[q][i];
      wx[i] = 0.5 * (R.b1 - R.a1) * c_gw[q][i];
      py[i] = 0.5 * (R.a2 + R.b2) + 0.5 * (R.b2 - R.a2) * c_gx[q][i];
      wy[i] = 0.5 * (R.b2 - R.a2) * c_gw[q][i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < q * p; i += kNT) {
      const int a = i / p, m = i % p;
      Lx[a * p + m] = lagrange_i(p, 2.0 * (px[a] - lx0) / lh - 1.0, m);
      Ly[a * p + m] = lagrange_i(p, 2.0 * (py[a] - ly0) / lh - 1.0, m);
    }
    for (int i = threadIdx.x; i < q * q; i += kNT) {
      const int a = i / q, c = i % q;
      double g, gx, gy;
      kernel_full(kernel, alpha, x - px[a], y - py[c], g, gx, gy);
      const double wt = wx[a] * wy[c];
      G[0][i] = g * wt; G[1][i] = gx * wt; G[2][i] = gy * wt;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * q * p; i += kNT) {
      const int f = i / (q * p), rem = i % (q * p);
      const int a = rem / p, j = rem % p;
      double s = 0.0;
      for (int c = 0; c < q; ++c) s += G[f][a * q + c] * Ly[c * p + j];
      H[f][a * p + j] = s;
    }
    __syncthreads();
    if (k < n) {
      for (int a = 0; a < q; ++a) {
        const double l = Lx[a * p + ki];
        a0 += l * H[0][a * p + kj];
        a1 += l * H[1][a * p + kj];
        a2 += l * H[2][a * p + kj];
      }
    }
    __syncthreads();
  }

  if (sdel > 0.0) {
    const double del = sdel;
    const int per_edge = kNAng * (kNRadPanels + 1) * kNRad;
    const int total = 4 * per_edge;
    for (int base = 0; base < total; base += kChunk) {
      if (threadIdx.x < kChunk) {
        const int idx = base + threadIdx.x;
        double w = 0.0, y1 = x, y2 = y;
        if (idx < total) {
          const int e = idx / per_edge;
          int rem = idx % per_edge;
          const int ia = rem / ((kNRadPanels + 1) * kNRad);
          rem %= (kNRadPanels + 1) * kNRad;
          const int kp = rem / kNRad, ir = rem % kNRad;
          const double nx = (e == 0) ? 1.0 : (e == 2 ? -1.0 : 0.0);
          const double ny = (e == 1) ? 1.0 : (e == 3 ? -1.0 : 0.0);
          const double phi = 0.25 * kPi * c_gx[kNAng][ia];
          const double wphi = 0.25 * kPi * c_gw[kNAng][ia];
          const double cp = cos(phi), sph = sin(phi);
          const double ex = cp * nx - sph * ny, ey = cp * ny + sph * nx;
          const double Rmax = del / cp;
          const double hi = ldexp(Rmax, -kp);
          const double lo = (kp == kNRadPanels) ? 0.0 : 0.5 * hi;
          const double rr = 0.5 * (lo + hi) + 0.5 * (hi - lo) * c_gx[kNRad][ir];
          w = wphi * 0.5 * (hi - lo) * c_gw[kNRad][ir] * rr;
          y1 = x + rr * ex;
          y2 = y + rr * ey;
        }
        double g = 0.0, gx = 0.0, gy = 0.0;
        if (w != 0.0) kernel_full(kernel, alpha, x - y1, y - y2, g, gx, gy);
        WG[0][threadIdx.x] = w * g; WG[1][threadIdx.x] = w * gx; WG[2][threadIdx.x] = w * gy;
        for (int m = 0; m < p; ++m) {
          L1[threadIdx.x * p + m] = lagrange_i(p, 2.0 * y1 / h - 1.0, m);
          L2[threadIdx.x * p + m] = lagrange_i(p, 2.0 * y2 / h - 1.0, m);
        }
      }
      __syncthreads();
      if (k < n) {
        for (int c = 0; c < kChunk; ++c) {
          const double l = L1[c * p + ki] * L2[c * p + kj];
          a0 += WG[0][c] * l; a1 += WG[1][c] * l; a2 += WG[2][c] * l;
        }
      }
      __syncthreads();
    }
  }
  if (k < n) {
    double* o = out + (size_t)pos * 3 * n * n;
    o[(size_t)(0 * n + t) * n + k] = a0;
    o[(size_t)(1 * n + t) * n + k] = a1;
    o[(size_t)(2 * n + t) * n + k] = a2;
  }
}

// ---------------------------------------------------------------- build-time GEMM
// C[b] (M x N, row stride ldc) = sum_k A[b](m,k) B[b](k,n) (+ beta*C), element strides given.
struct GemmDesc {
  int M, N, K;
  const double* A; long long am, ak, ab;
  const double* B; long long bk, bn, bb;
  double* C; long long cm, cn, cb;
  double beta;
};

__global__ void k_bgemm(GemmDesc d) {
  __shared__ double As[16][33];
  __shared__ double Bs[16][33];
  const int b = blockIdx.z;
  const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 256 threads, each 2x2
  double acc[2][2] = {{0, 0}, {0, 0}};
  const double* A = d.A + b * d.ab;
  const double* B = d.B + b * d.bb;
  for (int k0 = 0; k0 < d.K; k0 += 16) {
    for (int i = threadIdx.x; i < 16 * 32; i += 256) {
      const int kk = i / 32, mm = i % 32;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < d.M && gk < d.K) ? A[gm * d.am + gk * d.ak] : 0.0;
      const int gn = n0 + mm;
      Bs[kk][mm] = (gn < d.N && gk < d.K) ? B[gk * d.bk + gn * d.bn] : 0.0;
    }
    __syncthreads();
    for (int kk = 0; kk < 16; ++kk) {
      const double a0 = As[kk][ty * 2], a1 = As[kk][ty * 2 + 1];
      const double b0 = Bs[kk][tx * 2], b1 = Bs[kk][tx * 2 + 1];
      acc[0][0] += a0 * b0; acc[0][1] += a0 * b1; acc[1][0] += a1 * b0; acc[1][1] += a1 * b1;
    }
    __syncthreads();
  }
  double* C = d.C + b * d.cb;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      const int gm = m0 + ty * 2 + i, gn = n0 + tx * 2 + j;
      if (gm < d.M && gn < d.N) {
        double* c = C + gm * d.cm + gn * d.cn;
        *c = acc[i][j] + (d.beta != 0.0 ? d.beta * *c : 0.0);
      }
    }
}

cudaError_t bgemm(const GemmDesc& d, int batch, cudaStream_t s) {
  if (d.M <= 0 || d.N <= 0 || batch <= 0) return cudaSuccess;
  dim3 grid((d.N + 31) / 32, (d.M + 31) / 32, batch);
  k_bgemm<<<grid, 256, 0, s>>>(d);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- basis evaluation

struct ChanScale { double sK, sL; };

// Radial factors of channel-K local basis at z = alpha*rho with reference zr = alpha*r:
// RI[m] = I_m(z)/I_m(zr), and the gradient factors D1[m] = d/drho (I_m(alpha rho)/I_m(zr)),
// D2[m] = m/rho * I_m(alpha rho)/I_m(zr). Arrays of size P+2 scratch (ih, ihr).
__device__ void local_k_factors(double alpha, double rho, double r, int P, double* ih, double* ihr,
                                double* RI, double* D1, double* D2) {
  const double z = alpha * rho, zr = alpha * r;
  ihat(z, P + 1, ih);
  ihat(zr, P + 1, ihr);
  const double q = rho / r;
  double qm = 1.0;      // q^m
  double qm1 = 0.0;     // q^(m-1)
  for (int m = 0; m <= P; ++m) {
    RI[m] = qm * ih[m] / ihr[m];
    const double t2 = (alpha * alpha * rho / (4.0 * (m + 1.0))) * qm * ih[m + 1] / ihr[m];
    if (m == 0) {
      D1[0] = 2.0 * t2;  // I_0' = I_1
      D2[0] = 0.0;
    } else {
      const double t1 = (m / r) * qm1 * ih[m - 1] / ihr[m];
      D1[m] = t1 + t2;
      D2[m] = t1 - t2;
    }
    qm1 = qm;
    qm *= q;
  }
}

// Radial factors of channel-K multipole basis K_m(alpha rho)/K_m(alpha r):
// RK[m], and D1 = d/drho, D2 = m/rho * RK. Scratch kh (P+2), khr (P+2).
__device__ void mpole_k_factors(double alpha, double rho, double r, int P, double* kh, double* khr,
                                double* RK, double* D1, double* D2) {
  const double z = alpha * rho, zr = alpha * r;
  khat_scaled(z, P + 1, kh);
  khat_scaled(zr, P + 1, khr);
  const double e = exp(zr - z);
  const double q = r / rho;  // (zr/z)
  // RK[n] = K_n(z)/K_n(zr) = (zr/z)^n Khat_n(z)/Khat_n(zr)  (n >= 1); n = 0: Khat_0 ratio
  double qn = 1.0;
  double rk[64];
  for (int n2 = 0; n2 <= P + 1; ++n2) {
    rk[n2] = (n2 == 0 ? 1.0 : qn) * kh[n2] / khr[n2] * e;
    qn *= q;
    if (n2 == 0) qn = q;
  }
  // ratios at zr: K_{m+1}(zr)/K_m(zr), K_{m-1}(zr)/K_m(zr)
  for (int m = 0; m <= P; ++m) {
    RK[m] = rk[m];
    double up, dn;  // K_{m+1}(z)/K_m(zr), K_{m-1}(z)/K_m(zr)
    if (m == 0) {
      // K_1(zr)/K_0(zr) = Khat_1(zr)/(zr Khat_0(zr))
      up = rk[1] * khr[1] / (zr * khr[0]);
      dn = up;  // K_{-1} = K_1
      D1[0] = -alpha * up;  // K_0' = -K_1
      D2[0] = 0.0;
      continue;
    }
    // K_{m+1}(zr)/K_m(zr) = (2m/zr) Khat_{m+1}(zr)/Khat_m(zr)
    up = rk[m + 1] * (2.0 * m / zr) * khr[m + 1] / khr[m];
    if (m == 1) dn = rk[0] * khr[0] * zr / khr[1];
    else dn = rk[m - 1] * (zr / (2.0 * (m - 1.0))) * khr[m - 1] / khr[m];
    D1[m] = -0.5 * alpha * (dn + up);
    D2[m] = 0.5 * alpha * (up - dn);
  }
}

// Value and gradient of the cos/sin angular combination given radial factors.
// out[col] for col in [0, C): value; gx, gy likewise.
__device__ void angular_combine(int P, double th, const double* R, const double* D1, const double* D2,
                                double* v, double* gx, double* gy) {
  const double ct = cos(th), st = sin(th);
  for (int m = 0; m <= P; ++m) {
    const double cm = cos(m * th), sm = sin(m * th);
    v[m] = R[m] * cm;
    gx[m] = D1[m] * ct * cm + D2[m] * st * sm;
    gy[m] = D1[m] * st * cm - D2[m] * ct * sm;
    if (m > 0) {
      v[P + m] = R[m] * sm;
      gx[P + m] = D1[m] * ct * sm - D2[m] * st * cm;
      gy[P + m] = D1[m] * st * sm + D2[m] * ct * cm;
    }
  }
}

// Channel-L factors: local (rho/r)^m; multipole (r/rho)^m (m >= 1), log rho (m = 0).
__device__ void local_l_factors(double rho, double r, int P, double* R, double* D1, double* D2) {
  const double q = rho / r;
  double qm1 = 0.0, qm = 1.0;
  for (int m = 0; m <= P; ++m) {
    R[m] = qm;
    D1[m] = (m == 0) ? 0.0 : (m / r) * qm1;
    D2[m] = D1[m];
    qm1 = qm;
    qm *= q;
  }
}
__device__ void mpole_l_factors(double rho, double r, int P, double* R, double* D1, double* D2) {
  const double q = r / rho;
  double qm = q;
  R[0] = log(rho);
  D1[0] = 1.0 / rho;
  D2[0] = 0.0;
  for (int m = 1; m <= P; ++m) {
    R[m] = qm;
    D1[m] = -(m / rho) * qm;
    D2[m] = (m / rho) * qm;
    qm *= q;
  }
}

// Evaluate one channel's basis (values + gradient) at displacement (dx, dy) from the box centre.
// kind: 0 = multipole, 1 = local.  Outputs v, gx, gy of length 2P+1.
__device__ void eval_basis(int ch, int kind, double alpha, double r, int P, double dx, double dy, double* v,
                           double* gx, double* gy) {
  double a[64], b[64], R[64], D1[64], D2[64];
  const double rho = sqrt(dx * dx + dy * dy);
  const double th = (rho > 0.0) ? atan2(dy, dx) : 0.0;
  if (ch == 0) {
    if (kind == 1) local_k_factors(alpha, rho, r, P, a, b, R, D1, D2);
    else mpole_k_factors(alpha, rho, r, P, a, b, R, D1, D2);
  } else {
    if (kind == 1) local_l_factors(rho, r, P, R, D1, D2);
    else mpole_l_factors(rho, r, P, R, D1, D2);
  }
  angular_combine(P, th, R, D1, D2, v, gx, gy);
}

// L2T / M2T: rows (f, t) of a target leaf (centre-relative node coordinates), columns (ch, mode).
// Target leaf of side ht centred at (0,0); source box centre at (scx, scy) with reference radius rs.
// out layout: out[ch * stride_ch + (f*n + t) * C + mode].
__global__ void k_eval_basis_at_nodes(int p, int P, int nch, int kind, double alpha, double ht, double scx,
                                      double scy, double rs, const int* kact, double* out, long long stride_ch,
                                      int ldrow) {
  const int n = p * p;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int ch = blockIdx.y;
  if (t >= n || ch >= nch) return;
  if (ch == 0 && !kact[0]) return;
  const int C = 2 * P + 1;
  const double x = 0.5 * ht * c_gx[p][t % p], y = 0.5 * ht * c_gx[p][t / p];
  double v[128], gx[128], gy[128];
  eval_basis(ch, kind, alpha, rs, P, x - scx, y - scy, v, gx, gy);
  double* o = out + ch * stride_ch;
  for (int c = 0; c < C; ++c) {
    o[(size_t)(0 * n + t) * ldrow + c] = v[c];
    o[(size_t)(1 * n + t) * ldrow + c] = gx[c];
    o[(size_t)(2 * n + t) * ldrow + c] = gy[c];
  }
}

// Circle sampling for translation operators: for instance b, source basis (channel ch, kind) centred
// at src[b] with reference radius rs, sampled at Q points on the circle of radius rt about tgt[b].
// F[b][j][col].
struct CircleInst { double tcx, tcy, rt, scx, scy, rs; int ch, kind; };
__global__ void k_circle_sample(int P, int Q, double alpha, const CircleInst* inst, double* F) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (j >= Q) return;
  const CircleInst I = inst[b];
  const int C = 2 * P + 1;
  const double th = 2.0 * kPi * j / Q;
  const double x = I.tcx + I.rt * cos(th), y = I.tcy + I.rt * sin(th);
  double v[128], gx[128], gy[128];
  eval_basis(I.ch, I.kind, alpha, I.rs, P, x - I.scx, y - I.scy, v, gx, gy);
  double* o = F + ((size_t)b * Q + j) * C;
  for (int c = 0; c < C; ++c) o[c] = v[c];
}

// DFT matrix T[row][j]: rows = modes (0, cos 1..P, sin 1..P).
__global__ void k_dft_matrix(int P, int Q, double* T) {
  const int C = 2 * P + 1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= C * Q) return;
  const int row = idx / Q, j = idx % Q;
  const double th = 2.0 * kPi * j / Q;
  double v;
  if (row == 0) v = 1.0 / Q;
  else if (row <= P) v = 2.0 / Q * cos(row * th);
  else v = 2.0 / Q * sin((row - P) * th);
  T[idx] = v;
}

// S2M quadrature points over a leaf of side h centred at 0 (ns x ns sub-boxes, order q):
// Bm[pt][row] (row = ch*C + mode) and Lm[pt][k].
__global__ void k_s2m_points(int p, int P, int nch, int q, int ns, double alpha, double h, ChanScale sc,
                             int kact, double* Bm, double* Lm) {
  const int npt = q * q * ns * ns;
  const int pt = blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= npt) return;
  const int C = 2 * P + 1, E = nch * C, n = p * p;
  const int sub = pt / (q * q), rem = pt % (q * q);
  const int sx = sub % ns, sy = sub / ns, a = rem % q, c = rem / q;
  const double hs = h / ns;
  const double x0 = -0.5 * h + sx * hs, y0 = -0.5 * h + sy * hs;
  const double x = x0 + 0.5 * hs * (1.0 + c_gx[q][a]);
  const double y = y0 + 0.5 * hs * (1.0 + c_gx[q][c]);
  const double w = 0.25 * hs * hs * c_gw[q][a] * c_gw[q][c];
  const double r = h / sqrt(2.0);
  const double rho = sqrt(x * x + y * y);
  const double th = (rho > 0.0) ? atan2(y, x) : 0.0;
  double* B = Bm + (size_t)pt * E;
  // channel K: A_m = sK (eps_m/2pi) K_m(alpha r) I_m(alpha rho) {cos,sin}(m th)
  if (kact) {
    double ih[64], kh[64];
    ihat(alpha * rho, P, ih);
    khat_scaled(alpha * r, P, kh);
    const double ez = exp(-alpha * r);
    const double q1 = rho / r;
    double qm = 1.0;
    for (int m = 0; m <= P; ++m) {
      const double ki = (m == 0) ? kh[0] * ez * ih[0] : kh[m] * ez * ih[m] * qm / (2.0 * m);
      const double f = sc.sK * ((m == 0) ? 1.0 : 2.0) * ki * w;
      B[m] = f * cos(m * th);
      if (m > 0) B[P + m] = f * sin(m * th);
      qm *= q1;
    }
  } else {
    for (int m = 0; m < C; ++m) B[m] = 0.0;
  }
  if (nch == 2) {
    double* BL = B + C;
    BL[0] = sc.sL * w;
    const double q1 = rho / r;
    double qm = q1;
    for (int m = 1; m <= P; ++m) {
      const double f = -sc.sL / m * qm * w;
      BL[m] = f * cos(m * th);
      BL[P + m] = f * sin(m * th);
      qm *= q1;
    }
  }
  const double tx = 2.0 * x / h, ty = 2.0 * y / h;
  double lx[16], ly[16];
  for (int i = 0; i < p; ++i) { lx[i] = lagrange_i(p, tx, i); ly[i] = lagrange_i(p, ty, i); }
  double* L = Lm + (size_t)pt * n;
  for (int j = 0; j < p; ++j)
    for (int i = 0; i < p; ++i) L[j * p + i] = lx[i] * ly[j];
}

// S2L: kernel matrix from quadrature points over the coarse source leaf to target circle points.
// Points: source leaf [sx0, sx0+ss]^2 split 2x2, order q. Gm[b][j][pt] for instance b = (pos, ch).
struct S2LInst { double sx0, sy0, ss, tcx, tcy, rt; int ch; };
__global__ void k_s2l_kernel(int q, int Q, double alpha, ChanScale sc, const S2LInst* inst, double* Gm) {
  const int npt = 4 * q * q;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (idx >= npt * Q) return;
  const int j = idx / npt, pt = idx % npt;
  const S2LInst I = inst[b];
  const int sub = pt / (q * q), rem = pt % (q * q);
  const int a = rem % q, c = rem / q;
  const double hs = 0.5 * I.ss;
  const double x0 = I.sx0 + (sub % 2) * hs, y0 = I.sy0 + (sub / 2) * hs;
  const double yx = x0 + 0.5 * hs * (1.0 + c_gx[q][a]);
  const double yy = y0 + 0.5 * hs * (1.0 + c_gx[q][c]);
  const double w = 0.25 * hs * hs * c_gw[q][a] * c_gw[q][c];
  const double th = 2.0 * kPi * j / Q;
  const double xx = I.tcx + I.rt * cos(th), xy = I.tcy + I.rt * sin(th);
  const double r = sqrt((xx - yx) * (xx - yx) + (xy - yy) * (xy - yy));
  double g;
  if (I.ch == 0) {
    const double z = alpha * r;
    double k0s = 0.0, k1s = 0.0;
    if (z < 700.0) bessel_k01_scaled(z, k0s, k1s);
    g = (z < 700.0) ? sc.sK * k0s * exp(-z) : 0.0;
  } else {
    g = sc.sL * log(r);
  }
  Gm[((size_t)b * Q + j) * npt + pt] = g * w;
}

// Lagrange basis of the source leaf (side ss, points in its own frame) at the S2L points.
__global__ void k_s2l_lagrange(int p, int q, double* Lm) {
  const int npt = 4 * q * q, n = p * p;
  const int pt = blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= npt) return;
  const int sub = pt / (q * q), rem = pt % (q * q);
  const int a = rem % q, c = rem / q;
  // reference coordinates of the leaf [-1,1]^2, sub-box halves
  const double tx = -1.0 + (sub % 2) + 0.5 * (1.0 + c_gx[q][a]);
  const double ty = -1.0 + (sub / 2) + 0.5 * (1.0 + c_gx[q][c]);
  double lx[16], ly[16];
  for (int i = 0; i < p; ++i) { lx[i] = lagrange_i(p, tx, i); ly[i] = lagrange_i(p, ty, i); }
  for (int j = 0; j < p; ++j)
    for (int i = 0; i < p; ++i) Lm[(size_t)pt * n + j * p + i] = lx[i] * ly[j];
}

__global__ void k_set_charge_row(int C, int nch, double* m2m_lvl) {
  // channel L (index 1) multipole-to-multipole: the log coefficient is the total charge.
  if (nch < 2) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= 4 * C) return;
  double* row0 = m2m_lvl + (size_t)1 * C * 4 * C;  // channel 1, row 0
  row0[c] = (c % C == 0) ? 1.0 : 0.0;
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
  cudaError_t alloc(size_t bytes) { if (p) { cudaFree(p); p = nullptr; } return bytes ? cudaMalloc(&p, bytes) : cudaSuccess; }
  template <class T> T* as() const { return static_cast<T*>(p); }
};

#define TRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_last_cuda(e_); return e_ == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA; } } while (0)

int build_all(vp_tables_s* T, cudaStream_t s) {
  const int p = T->p, n = T->n, P = T->P, C = T->C, nch = T->nch, E = T->E, L = T->levels;
  const double alpha = T->alpha;
  const Positions& pos = positions();
  const ChanScale sc{T->kernel == VP_KERNEL_MHELMHOLTZ ? 0.5 / kPi : 0.5 / (kPi * alpha * alpha),
                     0.5 / (kPi * alpha * alpha)};

  // quadrature rules to constant memory
  {
    std::vector<double> gx((kMaxQ + 1) * kMaxQ, 0.0), gw((kMaxQ + 1) * kMaxQ, 0.0);
    for (int q : {p, 12, 16, 20, 24, 40}) host_gauss_legendre(q, &gx[q * kMaxQ], &gw[q * kMaxQ]);
    TRY(cudaMemcpyToSymbolAsync(c_gx, gx.data(), gx.size() * sizeof(double), 0, cudaMemcpyHostToDevice, s));
    TRY(cudaMemcpyToSymbolAsync(c_gw, gw.data(), gw.size() * sizeof(double), 0, cudaMemcpyHostToDevice, s));
    double bw[16] = {0};
    for (int i = 0; i < p; ++i) {
      double prod = 1.0;
      for (int j = 0; j < p; ++j) if (j != i) prod *= gx[p * kMaxQ + i] - gx[p * kMaxQ + j];
      bw[i] = 1.0 / prod;
    }
    TRY(cudaMemcpyToSymbolAsync(c_bw, bw, sizeof(bw), 0, cudaMemcpyHostToDevice, s));
  }

  const size_t nl = (size_t)L + 1;
  TRY(cudaMalloc(&T->near, nl * T->near_stride_lvl() * sizeof(double)));
  TRY(cudaMalloc(&T->s2m, nl * T->s2m_stride_lvl() * sizeof(double)));
  TRY(cudaMalloc(&T->l2t, nl * T->l2t_stride_lvl() * sizeof(double)));
  TRY(cudaMalloc(&T->m2m, nl * T->m2m_stride_lvl() * sizeof(double)));
  TRY(cudaMalloc(&T->l2l, nl * T->l2l_stride_lvl() * sizeof(double)));
  TRY(cudaMalloc(&T->m2l, nl * T->m2l_stride_lvl() * sizeof(double)));
  TRY(cudaMalloc(&T->m2t, nl * T->m2t_stride_lvl() * sizeof(double)));
  TRY(cudaMalloc(&T->s2l, nl * T->s2l_stride_lvl() * sizeof(double)));
  TRY(cudaMemsetAsync(T->s2m, 0, nl * T->s2m_stride_lvl() * sizeof(double), s));
  TRY(cudaMemsetAsync(T->l2t, 0, nl * T->l2t_stride_lvl() * sizeof(double), s));
  TRY(cudaMemsetAsync(T->m2m, 0, nl * T->m2m_stride_lvl() * sizeof(double), s));
  TRY(cudaMemsetAsync(T->l2l, 0, nl * T->l2l_stride_lvl() * sizeof(double), s));
  TRY(cudaMemsetAsync(T->m2l, 0, nl * T->m2l_stride_lvl() * sizeof(double), s));
  TRY(cudaMemsetAsync(T->m2t, 0, nl * T->m2t_stride_lvl() * sizeof(double), s));
  TRY(cudaMemsetAsync(T->s2l, 0, nl * T->s2l_stride_lvl() * sizeof(double), s));

  DevBuf d_err, d_geo, d_kact;
  TRY(d_err.alloc(sizeof(int)));
  TRY(cudaMemsetAsync(d_err.p, 0, sizeof(int), s));
  TRY(d_geo.alloc(sizeof(pos.near)));
  TRY(cudaMemcpyAsync(d_geo.p, pos.near, sizeof(pos.near), cudaMemcpyHostToDevice, s));
  TRY(d_kact.alloc(nl * sizeof(int)));
  TRY(cudaMemcpyAsync(d_kact.p, T->kactive.data(), nl * sizeof(int), cudaMemcpyHostToDevice, s));

  // near tables
  const int self_pos = pos.near_same[1][1];
  for (int l = 0; l <= L; ++l) {
    dim3 grid(n, kNearPos);
    k_near_table<<<grid, kNT, 0, s>>>(T->kernel, alpha, p, T->h(l), self_pos, d_geo.as<RelBox>(),
                                      T->near + l * T->near_stride_lvl(), d_err.as<int>());
    TRY(cudaGetLastError());
  }

  // S2M (leaf levels >= 2)
  {
    DevBuf Bm, Lm;
    const int q = 40;
    int max_ns = 1;
    for (int l = 2; l <= L; ++l) {
      const int ns = T->kactive[l] ? std::max(1, (int)std::ceil(alpha * T->h(l) / 10.0)) : 1;
      max_ns = std::max(max_ns, ns);
    }
    const size_t max_pts = (size_t)q * q * max_ns * max_ns;
    TRY(Bm.alloc(max_pts * E * sizeof(double)));
    TRY(Lm.alloc(max_pts * n * sizeof(double)));
    for (int l = 2; l <= L; ++l) {
      const int ns = T->kactive[l] ? std::max(1, (int)std::ceil(alpha * T->h(l) / 10.0)) : 1;
      const int npt = q * q * ns * ns;
      k_s2m_points<<<(npt + 127) / 128, 128, 0, s>>>(p, P, nch, q, ns, alpha, T->h(l), sc, T->kactive[l],
                                                     Bm.as<double>(), Lm.as<double>());
      TRY(cudaGetLastError());
      GemmDesc d{E, n, npt, Bm.as<double>(), 1, E, 0, Lm.as<double>(), n, 1, 0,
                 T->s2m + l * T->s2m_stride_lvl(), n, 1, 0, 0.0};
      TRY(bgemm(d, 1, s));
    }
  }

  // L2T (leaf levels >= 2), M2T (target level l >= 1, source level l+1)
  for (int l = 2; l <= L; ++l) {
    const double r = T->h(l) / std::sqrt(2.0);
    dim3 grid((n + 127) / 128, nch);
    // l2t layout [3n][E]: channel ch columns at offset ch*C
    k_eval_basis_at_nodes<<<grid, 128, 0, s>>>(p, P, nch, 1, alpha, T->h(l), 0.0, 0.0, r,
                                               d_kact.as<int>() + l, T->l2t + l * T->l2t_stride_lvl(), C, E);
    TRY(cudaGetLastError());
  }
  for (int l = 1; l < L; ++l) {
    const double h = T->h(l);
    const double rs = T->h(l + 1) / std::sqrt(2.0);
    for (int w = 0; w < kWPos; ++w) {
      const RelBox& b = pos.w[w];
      // target leaf centred at 0: source centre relative to target centre
      const double scx = (b.ox + 0.5 * b.s - 0.5) * h, scy = (b.oy + 0.5 * b.s - 0.5) * h;
      dim3 grid((n + 127) / 128, nch);
      k_eval_basis_at_nodes<<<grid, 128, 0, s>>>(p, P, nch, 0, alpha, h, scx, scy, rs, d_kact.as<int>() + l + 1,
                                                 T->m2t + l * T->m2t_stride_lvl() + w * T->m2t_stride_pos(),
                                                 T->m2t_stride_ch(), C);
      TRY(cudaGetLastError());
    }
  }

  // translation operators by circle sampling
  const int Q = 512;
  DevBuf dT;
  TRY(dT.alloc((size_t)C * Q * sizeof(double)));
  k_dft_matrix<<<(C * Q + 255) / 256, 256, 0, s>>>(P, Q, dT.as<double>());
  TRY(cudaGetLastError());
  {
    DevBuf F, dinst;
    const int max_inst = kVOff * nch;
    TRY(F.alloc((size_t)max_inst * Q * C * sizeof(double)));
    TRY(dinst.alloc(max_inst * sizeof(CircleInst)));
    std::vector<CircleInst> inst;
    auto run = [&](double* out_base, long long out_stride_inst, int ldc) -> int {
      const int nb = (int)inst.size();
      if (nb == 0) return VP_OK;
      TRY(cudaMemcpyAsync(dinst.p, inst.data(), nb * sizeof(CircleInst), cudaMemcpyHostToDevice, s));
      dim3 grid((Q + 127) / 128, nb);
      k_circle_sample<<<grid, 128, 0, s>>>(P, Q, alpha, dinst.as<CircleInst>(), F.as<double>());
      TRY(cudaGetLastError());
      // out[b] (C x C, row stride ldc) = T (C x Q) * F[b] (Q x C)
      GemmDesc d{C, C, Q, dT.as<double>(), Q, 1, 0, F.as<double>(), C, 1, (long long)Q * C,
                 out_base, ldc, 1, out_stride_inst, 0.0};
      TRY(bgemm(d, nb, s));
      // the stream must not reuse `inst` host memory before the copy: synchronise
      TRY(cudaStreamSynchronize(s));
      return VP_OK;
    };
    for (int l = 2; l <= L; ++l) {
      const double h = T->h(l), r = h / std::sqrt(2.0);
      // M2L: target centre 0, source centre (dx h, dy h); out m2l[l][off][ch]
      for (int ch = 0; ch < nch; ++ch) {
        if (ch == 0 && !T->kactive[l]) continue;
        inst.clear();
        for (int o = 0; o < kVOff; ++o) inst.push_back({0.0, 0.0, r, pos.v_dx[o] * h, pos.v_dy[o] * h, r, ch, 0});
        const int rc = run(T->m2l + l * T->m2l_stride_lvl() + ch * T->m2l_stride_ch(), T->m2l_stride_off(), C);
        if (rc) return rc;
      }
    }
    for (int l = 2; l < L; ++l) {
      const double h = T->h(l), r = h / std::sqrt(2.0), rc_ = T->h(l + 1) / std::sqrt(2.0);
      for (int ch = 0; ch < nch; ++ch) {
        if (ch == 0 && !T->kactive[l]) continue;
        // M2M: parent circle (centre 0, radius r), child multipole at quadrant centre, columns q*C..
        inst.clear();
        for (int qd = 0; qd < 4; ++qd) {
          const double cx = ((qd % 2) - 0.5) * 0.5 * h, cy = ((qd / 2) - 0.5) * 0.5 * h;
          inst.push_back({0.0, 0.0, r, cx, cy, rc_, ch, 0});
        }
        int rc = run(T->m2m + l * T->m2m_stride_lvl() + ch * T->m2m_stride_ch(), C, 4 * C);
        if (rc) return rc;
        // L2L: child circle (centre quadrant, radius r_child), parent local at 0; out l2l[l][q][ch]
        inst.clear();
        for (int qd = 0; qd < 4; ++qd) {
          const double cx = ((qd % 2) - 0.5) * 0.5 * h, cy = ((qd / 2) - 0.5) * 0.5 * h;
          inst.push_back({cx, cy, rc_, 0.0, 0.0, r, ch, 1});
        }
        rc = run(T->l2l + l * T->l2l_stride_lvl() + ch * T->l2l_stride_ch(), T->l2l_stride_q(), C);
        if (rc) return rc;
      }
      k_set_charge_row<<<(4 * C + 127) / 128, 128, 0, s>>>(C, nch, T->m2m + l * T->m2m_stride_lvl());
      TRY(cudaGetLastError());
    }
  }

  // S2L (target level l >= 2, source leaf level l-1)
  {
    const int q = 24, Qs = 256;
    const int npt = 4 * q * q;
    DevBuf dTs, Gm, Lm, V, dinst;
    TRY(dTs.alloc((size_t)C * Qs * sizeof(double)));
    k_dft_matrix<<<(C * Qs + 255) / 256, 256, 0, s>>>(P, Qs, dTs.as<double>());
    TRY(cudaGetLastError());
    const int max_inst = kXPos * nch;
    TRY(Gm.alloc((size_t)max_inst * Qs * npt * sizeof(double)));
    TRY(Lm.alloc((size_t)npt * n * sizeof(double)));
    TRY(V.alloc((size_t)max_inst * Qs * n * sizeof(double)));
    TRY(dinst.alloc(max_inst * sizeof(S2LInst)));
    k_s2l_lagrange<<<(npt + 127) / 128, 128, 0, s>>>(p, q, Lm.as<double>());
    TRY(cudaGetLastError());
    std::vector<S2LInst> inst;
    for (int l = 2; l <= L; ++l) {
      const double h = T->h(l), r = h / std::sqrt(2.0);
      inst.clear();
      for (int xp = 0; xp < kXPos; ++xp)
        for (int ch = 0; ch < nch; ++ch) {
          if (ch == 0 && !T->kactive[l]) continue;
          const RelBox& b = pos.x[xp];
          inst.push_back({b.ox * h, b.oy * h, b.s * h, 0.5 * h, 0.5 * h, r, ch});
        }
      const int nb = (int)inst.size();
      if (nb == 0) continue;
      TRY(cudaMemcpyAsync(dinst.p, inst.data(), nb * sizeof(S2LInst), cudaMemcpyHostToDevice, s));
      dim3 grid((npt * Qs + 255) / 256, nb);
      k_s2l_kernel<<<grid, 256, 0, s>>>(q, Qs, alpha, sc, dinst.as<S2LInst>(), Gm.as<double>());
      TRY(cudaGetLastError());
      // V[b] (Qs x n) = Gm[b] (Qs x npt) * Lm (npt x n)
      GemmDesc d1{Qs, n, npt, Gm.as<double>(), npt, 1, (long long)Qs * npt, Lm.as<double>(), n, 1, 0,
                  V.as<double>(), n, 1, (long long)Qs * n, 0.0};
      TRY(bgemm(d1, nb, s));
      // S2L[b] (C x n) = Ts (C x Qs) * V[b]; scatter instance b to s2l[l][xp][ch]
      int b = 0;
      for (int xp = 0; xp < kXPos; ++xp)
        for (int ch = 0; ch < nch; ++ch) {
          if (ch == 0 && !T->kactive[l]) continue;
          GemmDesc d2{C, n, Qs, dTs.as<double>(), Qs, 1, 0, V.as<double>() + (size_t)b * Qs * n, n, 1, 0,
                      T->s2l + l * T->s2l_stride_lvl() + xp * T->s2l_stride_pos() + ch * T->s2l_stride_ch(), n, 1,
                      0, 0.0};
          TRY(bgemm(d2, 1, s));
          ++b;
        }
      TRY(cudaStreamSynchronize(s));
    }
  }

  TRY(cudaStreamSynchronize(s));
  int herr = 0;
  TRY(cudaMemcpy(&herr, d_err.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) return VP_ERR_CUDA;
  return VP_OK;
}

}  // namespace

void gauss_legendre_host(int n, double* x, double* w) { host_gauss_legendre(n, x, w); }

}  // namespace vp

namespace vp {
namespace {
// One thread per argument: the device special functions, for checks against reference values.
__global__ void k_special(int which, int nmax, int count, const double* z, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double v[kSpecialMaxOrder + 1];
  const double x = z[i];
  if (which == 0) {
    bessel_k01_scaled(x, v[0], v[1]);
    out[i] = v[0];
    out[count + i] = v[1];
    return;
  }
  if (which == 1) khat_scaled(x, nmax, v);
  else ihat(x, nmax, v);
  for (int n = 0; n <= nmax; ++n) out[(long long)n * count + i] = v[n];
}
}  // namespace
}  // namespace vp

extern "C" int vp_special(int which, int nmax, int count, const double* z, double* out, void* stream) {
  if (which < 0 || which > 2 || count < 0 || (count > 0 && (!z || !out)) ||
      (which > 0 && (nmax < 1 || nmax > vp::kSpecialMaxOrder)))
    return VP_ERR_ARG;
  if (count == 0) return VP_OK;
  vp::k_special<<<(count + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(which, nmax, count, z, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    vp::set_last_cuda(e);
    return VP_ERR_CUDA;
  }
  return VP_OK;
}

extern "C" int vp_tables_build(int kernel, double alpha, int p, int levels, double root_side, int order,
                               int precision, void* stream, vp_tables* out) {
  if (!out) return VP_ERR_ARG;
  *out = nullptr;
  if ((kernel != VP_KERNEL_MHELMHOLTZ && kernel != VP_KERNEL_MBIHARMONIC) || !(alpha > 0.0) || !std::isfinite(alpha) ||
      p < 2 || p > 16 || levels < 0 || levels > 20 || !(root_side > 0.0) || !std::isfinite(root_side) || order < 4 ||
      order > 60 || (precision != VP_PREC_FP64 && precision != VP_PREC_SPLIT))
    return VP_ERR_ARG;
  std::unique_ptr<vp_tables_s> T(new (std::nothrow) vp_tables_s());
  if (!T) return VP_ERR_OOM;
  T->kernel = kernel; T->alpha = alpha; T->p = p; T->n = p * p; T->P = order; T->C = 2 * order + 1;
  T->nch = (kernel == VP_KERNEL_MBIHARMONIC) ? 2 : 1; T->E = T->nch * T->C; T->levels = levels;
  T->precision = precision; T->side = root_side;
  T->kactive.assign(levels + 1, 0);
  for (int l = 0; l <= levels; ++l) T->kactive[l] = (alpha * T->h(l) <= 60.0) ? 1 : 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = vp::build_all(T.get(), s);
  if (rc == VP_OK && precision == VP_PREC_SPLIT) rc = vp::build_split(T.get(), s);
  if (rc != VP_OK) {
    vp_tables_free(T.release());
    return rc;
  }
  *out = T.release();
  return VP_OK;
}

extern "C" void vp_tables_free(vp_tables t) {
  if (!t) return;
  vp::free_split_tables(t);
  for (void* ptr : {(void*)t->near, (void*)t->s2m, (void*)t->l2t, (void*)t->m2m, (void*)t->l2l, (void*)t->m2l,
                    (void*)t->m2t, (void*)t->s2l})
    if (ptr) cudaFree(ptr);
  delete t;
}
