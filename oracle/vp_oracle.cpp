// Direct-quadrature oracle for the free-space volume potential on a quadtree.
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product path may load or call this
// file; only the tests, the smoke check and the CPU-baseline leg of the bench do.
// It shares no code with the CUDA library.
//
// What it computes (paper Sec. 2.1, Eq. vol_pot, in its scalar form, restricted
// to the box that the leaves tile): for each target x,
//
//     u(x)      = sum over leaves L of  int_L G(x - y) f_L(y) dy
//     grad u(x) = sum over leaves L of  int_L grad_x G(x - y) f_L(y) dy
//
// where f_L is the degree-(p-1) tensor Lagrange interpolant of the nodal values
// on leaf L at p x p Gauss-Legendre nodes, and G is one of
//
//     G1(r) = K0(alpha r) / (2 pi)                       (alpha^2 - Laplacian)
//     G2(r) = (K0(alpha r) + log r) / (2 pi alpha^2)     (Laplacian (alpha^2 - Laplacian))
//
// G2 is minus the modified-biharmonic Green's function of Sec. 2 (Eq. modbiharm);
// it equals Q0(r)/(2 pi alpha^2) with Q0 of Sec. 3.2.1 (Eq. Q0).
//
// Quadrature (plain, slow, a-priori error control):
//  * a leaf (or piece of one) whose distance from x is at least its longest side
//    is integrated with a tensor Gauss-Legendre rule whose order grows as the
//    distance ratio shrinks;
//  * a closer piece is split (in two along a long side, else in four) until
//    every piece is far in that sense;
//  * the leaf that contains x: the square centred at x touching the nearest leaf
//    edge is integrated in polar coordinates about x (four triangles, Gauss-
//    Legendre in angle, geometrically graded Gauss-Legendre panels in radius),
//    which absorbs the log r and 1/r behaviour of G and grad G; the rest of the
//    leaf is a union of rectangles at positive distance from x, handled above.
// Bessel functions come from libstdc++ (std::cyl_bessel_k), log from libm.
// Parity is pinned by the tests against closed forms (radial Gaussian sources,
// manufactured solutions, constant sources) and against brute force.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr double kPi = 3.14159265358979323846;

struct Rule { std::vector<double> x, w; };

// Gauss-Legendre nodes/weights on [-1,1] by Newton's method on the three-term
// recurrence for P_n (textbook construction, ascending order).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0); w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double t = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
      if (n == 1) { p1 = t; p0 = 1.0; }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
      double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    double p0 = 1.0, p1 = t;
    for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
    if (n == 1) { p1 = t; p0 = 1.0; }
    dp = n * (t * p1 - p0) / (t * t - 1.0);
    x[n - 1 - i] = t;
    w[n - 1 - i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

struct Ctx {
  int kernel; double alpha; int p;
  std::vector<double> xi, bw;         // interpolation nodes and barycentric weights
  Rule gl[33];                        // tensor rules by order
  Rule ang, rad;                      // polar rules
  int n_rad_panels;
};

void init_ctx(Ctx& c, int kernel, double alpha, int p) {
  c.kernel = kernel; c.alpha = alpha; c.p = p;
  std::vector<double> w;
  gauss_legendre(p, c.xi, w);
  c.bw.assign(p, 1.0);
  for (int i = 0; i < p; ++i) {
    double prod = 1.0;
    for (int j = 0; j < p; ++j) if (j != i) prod *= (c.xi[i] - c.xi[j]);
    c.bw[i] = 1.0 / prod;
  }
  for (int q : {12, 14, 16, 18, 20, 24, 32}) gauss_legendre(q, c.gl[q].x, c.gl[q].w);
  gauss_legendre(24, c.ang.x, c.ang.w);
  gauss_legendre(14, c.rad.x, c.rad.w);
  c.n_rad_panels = 22;
}

// Lagrange basis values l_i(t), i < p, at t in reference coordinates.
inline void lagrange(const Ctx& c, double t, double* out) {
  const int p = c.p;
  for (int i = 0; i < p; ++i) {
    if (t == c.xi[i]) { for (int k = 0; k < p; ++k) out[k] = (k == i) ? 1.0 : 0.0; return; }
  }
  double s = 0.0;
  for (int i = 0; i < p; ++i) { out[i] = c.bw[i] / (t - c.xi[i]); s += out[i]; }
  for (int i = 0; i < p; ++i) out[i] /= s;
}

// G, dG/dx, dG/dy for displacement d = x - y.
inline void kernel_eval(const Ctx& c, double dx, double dy, double& g, double& gx, double& gy) {
  const double r = std::sqrt(dx * dx + dy * dy);
  const double z = c.alpha * r;
  double k0 = 0.0, k1 = 0.0;
  if (z < 700.0) { k0 = std::cyl_bessel_k(0.0, z); k1 = std::cyl_bessel_k(1.0, z); }
  double gp;
  if (c.kernel == 0) {
    g = k0 / (2.0 * kPi);
    gp = -c.alpha * k1 / (2.0 * kPi);
  } else {
    const double s = 1.0 / (2.0 * kPi * c.alpha * c.alpha);
    g = (k0 + std::log(r)) * s;
    gp = (-c.alpha * k1 + 1.0 / r) * s;
  }
  gx = gp * dx / r;
  gy = gp * dy / r;
}

struct Leaf { double x0, y0, h; const double* f; double fmax; };
struct Rect { double a1, b1, a2, b2; };
struct Acc { double u = 0, ux = 0, uy = 0; };

inline double rect_dist(const Rect& R, double x, double y) {
  double dx = std::max(std::max(R.a1 - x, 0.0), x - R.b1);
  double dy = std::max(std::max(R.a2 - y, 0.0), y - R.b2);
  return std::sqrt(dx * dx + dy * dy);
}

// f_L at an arbitrary point (tensor Lagrange interpolant of the leaf values).
inline double interp(const Ctx& c, const Leaf& L, double y1, double y2, double* l1, double* l2) {
  lagrange(c, 2.0 * (y1 - L.x0) / L.h - 1.0, l1);
  lagrange(c, 2.0 * (y2 - L.y0) / L.h - 1.0, l2);
  double s = 0.0;
  for (int j = 0; j < c.p; ++j) {
    double t = 0.0;
    for (int i = 0; i < c.p; ++i) t += L.f[j * c.p + i] * l1[i];
    s += t * l2[j];
  }
  return s;
}

int order_for(double eta) {
  if (eta < 2.0) return 20;
  if (eta < 4.0) return 18;
  if (eta < 8.0) return 16;
  return 14;
}

// Tensor Gauss-Legendre over a rectangle at positive distance from x.
void tensor_rule(const Ctx& c, const Leaf& L, const Rect& R, double x, double y, int q, Acc& acc) {
  const Rule& g = c.gl[q];
  const int p = c.p;
  double Lx[32 * 32], Ly[32 * 32], tmp[32 * 32];
  double px[32], py[32], wx[32], wy[32];
  for (int a = 0; a < q; ++a) {
    px[a] = 0.5 * (R.a1 + R.b1) + 0.5 * (R.b1 - R.a1) * g.x[a];
    wx[a] = 0.5 * (R.b1 - R.a1) * g.w[a];
    py[a] = 0.5 * (R.a2 + R.b2) + 0.5 * (R.b2 - R.a2) * g.x[a];
    wy[a] = 0.5 * (R.b2 - R.a2) * g.w[a];
    lagrange(c, 2.0 * (px[a] - L.x0) / L.h - 1.0, &Lx[a * p]);
    lagrange(c, 2.0 * (py[a] - L.y0) / L.h - 1.0, &Ly[a * p]);
  }
  // tmp[a][j] = sum_i Lx[a][i] f[j][i]
  for (int a = 0; a < q; ++a)
    for (int j = 0; j < p; ++j) {
      double s = 0.0;
      for (int i = 0; i < p; ++i) s += Lx[a * p + i] * L.f[j * p + i];
      tmp[a * p + j] = s;
    }
  for (int a = 0; a < q; ++a)
    for (int b = 0; b < q; ++b) {
      double fv = 0.0;
      for (int j = 0; j < p; ++j) fv += tmp[a * p + j] * Ly[b * p + j];
      double gg, gx, gy;
      kernel_eval(c, x - px[a], y - py[b], gg, gx, gy);
      const double wt = wx[a] * wy[b] * fv;
      acc.u += wt * gg; acc.ux += wt * gx; acc.uy += wt * gy;
    }
}

// Polar coordinates about x over the square of half-width d centred at x:
// four right isosceles triangles, angle in [-pi/4, pi/4] from each edge normal.
void polar_square(const Ctx& c, const Leaf& L, double x, double y, double d, Acc& acc) {
  double l1[64], l2[64];
  const double nx[4] = {1, 0, -1, 0}, ny[4] = {0, 1, 0, -1};
  const int K = c.n_rad_panels;
  for (int e = 0; e < 4; ++e) {
    const double tx = -ny[e], ty = nx[e];
    for (size_t ia = 0; ia < c.ang.x.size(); ++ia) {
      const double phi = 0.25 * kPi * c.ang.x[ia];
      const double wphi = 0.25 * kPi * c.ang.w[ia];
      const double ex = std::cos(phi) * nx[e] + std::sin(phi) * tx;
      const double ey = std::cos(phi) * ny[e] + std::sin(phi) * ty;
      const double Rmax = d / std::cos(phi);
      // radial panels [R 2^-(k+1), R 2^-k], k = 0..K-1, and [0, R 2^-K]
      for (int k = 0; k <= K; ++k) {
        double hi = Rmax * std::ldexp(1.0, -k);
        double lo = (k == K) ? 0.0 : 0.5 * hi;
        for (size_t ir = 0; ir < c.rad.x.size(); ++ir) {
          const double r = 0.5 * (lo + hi) + 0.5 * (hi - lo) * c.rad.x[ir];
          const double wr = 0.5 * (hi - lo) * c.rad.w[ir];
          const double y1 = x + r * ex, y2 = y + r * ey;
          const double fv = interp(c, L, y1, y2, l1, l2);
          double gg, gx, gy;
          kernel_eval(c, x - y1, y - y2, gg, gx, gy);
          const double wt = wphi * wr * r * fv;
          acc.u += wt * gg; acc.ux += wt * gx; acc.uy += wt * gy;
        }
      }
    }
  }
}

// Integral over one leaf. Returns 0, or -1 if x lies on the leaf boundary.
int leaf_integral(const Ctx& c, const Leaf& L, double x, double y, Acc& acc) {
  std::vector<Rect> stack;
  Rect full{L.x0, L.x0 + L.h, L.y0, L.y0 + L.h};
  const bool inside = x >= full.a1 && x <= full.b1 && y >= full.a2 && y <= full.b2;
  if (inside) {
    const double d = std::min(std::min(x - full.a1, full.b1 - x), std::min(y - full.a2, full.b2 - y));
    if (!(d > 0.0)) return -1;
    polar_square(c, L, x, y, d, acc);
    // remainder: left and right strips (full height), bottom and top pieces of the middle column
    Rect rl{full.a1, x - d, full.a2, full.b2}, rr{x + d, full.b1, full.a2, full.b2};
    Rect rb{x - d, x + d, full.a2, y - d}, rt{x - d, x + d, y + d, full.b2};
    for (const Rect& R : {rl, rr, rb, rt})
      if (R.b1 - R.a1 > 0.0 && R.b2 - R.a2 > 0.0) stack.push_back(R);
  } else {
    stack.push_back(full);
  }
  while (!stack.empty()) {
    Rect R = stack.back(); stack.pop_back();
    const double w = R.b1 - R.a1, h = R.b2 - R.a2;
    const double s = std::max(w, h);
    const double dist = rect_dist(R, x, y);
    if (dist >= s) { tensor_rule(c, L, R, x, y, order_for(dist / s), acc); continue; }
    if (!(dist > 0.0)) return -1;
    if (w > 2.0 * h) {
      const double m = 0.5 * (R.a1 + R.b1);
      stack.push_back({R.a1, m, R.a2, R.b2}); stack.push_back({m, R.b1, R.a2, R.b2});
    } else if (h > 2.0 * w) {
      const double m = 0.5 * (R.a2 + R.b2);
      stack.push_back({R.a1, R.b1, R.a2, m}); stack.push_back({R.a1, R.b1, m, R.b2});
    } else {
      const double m1 = 0.5 * (R.a1 + R.b1), m2 = 0.5 * (R.a2 + R.b2);
      stack.push_back({R.a1, m1, R.a2, m2}); stack.push_back({m1, R.b1, R.a2, m2});
      stack.push_back({R.a1, m1, m2, R.b2}); stack.push_back({m1, R.b1, m2, R.b2});
    }
  }
  return 0;
}

}  // namespace

extern "C" {

// Gauss-Legendre rule of order n on [-1, 1]; x, w have room for n values.
int ora_gauss_legendre(int n, double* x, double* w) {
  if (n < 1 || n > 64 || !x || !w) return -1;
  std::vector<double> xs, ws;
  gauss_legendre(n, xs, ws);
  std::memcpy(x, xs.data(), n * sizeof(double));
  std::memcpy(w, ws.data(), n * sizeof(double));
  return 0;
}

// Kernel G(r) and dG/dr for n radii (kernel 0: G1, kernel 1: G2).
int ora_kernel(int kernel, double alpha, int n, const double* r, double* g, double* dg) {
  if ((kernel != 0 && kernel != 1) || !(alpha > 0.0) || n < 0) return -1;
  Ctx c; init_ctx(c, kernel, alpha, 2);
  for (int i = 0; i < n; ++i) {
    double gg, gx, gy;
    kernel_eval(c, r[i], 0.0, gg, gx, gy);
    g[i] = gg; dg[i] = gx;
  }
  return 0;
}

// Volume potential u and grad u at n_targets points (tx, ty).
//   kernel 0: G1, kernel 1: G2; alpha > 0; 2 <= p <= 20.
//   Leaves: (level, ix, iy) in the root box centred at (cx, cy) with side `side`;
//   f holds n_leaves*p*p nodal values, node (i, j) of a leaf at j*p+i.
//   Returns 0, -1 on bad arguments, -2 if a target lies on a leaf boundary.
//   nthreads <= 0 uses the OpenMP default.
int ora_volume_potential(int kernel, double alpha, int p, double cx, double cy, double side,
                         int n_leaves, const int32_t* level, const int32_t* ix, const int32_t* iy,
                         const double* f, int n_targets, const double* tx, const double* ty,
                         double* u, double* ux, double* uy, int nthreads) {
  if ((kernel != 0 && kernel != 1) || !(alpha > 0.0) || p < 2 || p > 20 || n_leaves < 0 || n_targets < 0)
    return -1;
  Ctx c; init_ctx(c, kernel, alpha, p);
  std::vector<Leaf> leaves(n_leaves);
  for (int k = 0; k < n_leaves; ++k) {
    const double h = side / std::ldexp(1.0, level[k]);
    double fm = 0.0;
    for (int m = 0; m < p * p; ++m) fm = std::max(fm, std::fabs(f[(size_t)k * p * p + m]));
    leaves[k] = {cx - 0.5 * side + ix[k] * h, cy - 0.5 * side + iy[k] * h, h, f + (size_t)k * p * p, fm};
  }
  int status = 0;
#ifdef _OPENMP
  const int nt = nthreads > 0 ? nthreads : omp_get_num_procs();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
  for (int t = 0; t < n_targets; ++t) {
    Acc acc;
    for (int k = 0; k < n_leaves; ++k) {
      if (leaves[k].fmax == 0.0) continue;
      if (leaf_integral(c, leaves[k], tx[t], ty[t], acc) != 0) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
        status = -2;
      }
    }
    u[t] = acc.u; ux[t] = acc.ux; uy[t] = acc.uy;
  }
  return status;
}

int ora_num_threads(void) {
#ifdef _OPENMP
  return omp_get_num_procs();
#else
  return 1;
#endif
}

}  // extern "C"
