// Modified Stokes kernels shared by the boundary integral equation (bie.cu) and the layer-potential
// evaluation on the volume tree (layer.cu): the scalar functions of the stokeslet and stresslet
// (App. B, evaluated with the power series of App. C for small alpha r) and the double-layer kernel
// of Sec. 2.2 (Eq. dbl_lyr_ker).
#pragma once

#include <cuda_runtime.h>

#include "special.cuh"

namespace vp {

// Series coefficients of App. C: k0(z, n), k1(z, n) for L = log(z/2), with psi(n+1) by recursion.
struct KSeries {
  double k0[24], k1[24];
};
__device__ inline void k_series(double z, KSeries& s) {
  const double L = log(0.5 * z);
  double psi1 = -kEulerGamma;  // psi(n+1)
  double f = 1.0;              // 1 / (4^n (n!)^2)
  double g = 0.25;             // 1 / (4^(n+1) n! (n+1)!)
  for (int n = 0; n < 24; ++n) {
    const double psi2 = psi1 + 1.0 / (n + 1);
    s.k0[n] = (psi1 - L) * f;
    s.k1[n] = (2.0 * L - psi1 - psi2) * g;
    f /= 4.0 * (n + 1.0) * (n + 1.0);
    g /= 4.0 * (n + 1.0) * (n + 2.0);
    psi1 = psi2;
  }
}

// Stresslet and stokeslet scalar functions of App. B: T1, T2, T3, S1, S2 at z = alpha r.
__device__ inline void stress_funcs(double z, double& T1, double& T2, double& T3, double& S1, double& S2) {
  const double ip = 1.0 / kPi;
  if (z <= 1.5) {
    KSeries s;
    k_series(z, s);
    const double z2 = z * z;
    double a1 = 0.0, a2 = 0.0, a3 = 0.0, b1 = 0.0, b2 = 0.0;
    double zp = 1.0;  // z^(2n)
    for (int n = 0; n < 23; ++n) {
      // T1 = -(1/2pi) sum_{n>=1} (2k0(n) + 4k1(n) + k1(n-1)) z^(2n-2)
      if (n >= 1) a1 += (2.0 * s.k0[n] + 4.0 * s.k1[n] + s.k1[n - 1]) * zp / z2;
      // T2 = (1/pi)[-z^-4 + z^-2/8 + sum_{n>=2} (4k0(n) + 8k1(n) + k1(n-1)) z^(2n-4)]
      if (n >= 2) a2 += (4.0 * s.k0[n] + 8.0 * s.k1[n] + s.k1[n - 1]) * zp / (z2 * z2);
      // T3 = (1/2pi) sum_{n>=0} k1(n) z^(2n)
      a3 += s.k1[n] * zp;
      // S1 = (1/2pi) sum_{n>=0} (k0(n) + k1(n)) z^(2n)
      b1 += (s.k0[n] + s.k1[n]) * zp;
      // S2 = -(1/2pi)[-z^-2/2 + sum_{n>=1} (k0(n) + 2k1(n)) z^(2n-2)]
      if (n >= 1) b2 += (s.k0[n] + 2.0 * s.k1[n]) * zp / z2;
      zp *= z2;
    }
    T1 = -0.5 * ip * a1;
    T2 = ip * (-1.0 / (z2 * z2) + 0.125 / z2 + a2);
    T3 = 0.5 * ip * a3;
    S1 = 0.5 * ip * b1;
    S2 = -0.5 * ip * (-0.5 / z2 + b2);
  } else {
    double k0s, k1s;
    bessel_k01_scaled(z, k0s, k1s);
    const double e = (z < 700.0) ? exp(-z) : 0.0;
    const double K0 = k0s * e, K1 = k1s * e;
    const double z2 = z * z, z4 = z2 * z2;
    T1 = -(2.0 * z2 * K0 + (z2 + 4.0) * z * K1 - 4.0) / (2.0 * kPi * z4);
    T2 = (4.0 * z2 * K0 + (z2 + 8.0) * z * K1 - 8.0) / (kPi * z4 * z2);
    T3 = (z * K1 - 1.0) / (2.0 * kPi * z2);
    S1 = (z2 * K0 + z * K1 - 1.0) / (2.0 * kPi * z2);
    S2 = -(z2 * K0 + 2.0 * z * K1 - 2.0) / (2.0 * kPi * z4);
  }
}

// Double-layer kernel D_ab(x, y) for r = x - y, normal n = n(y):
// D_ab = -a^2 T1 (n_a r_b + n_b r_a + d_ab r.n) - a^4 T2 r_a r_b r.n - a^2 T3 r_a n_b.
__device__ inline void dl_kernel(double alpha, double rx, double ry, double nx, double ny, double D[4]) {
  const double r = sqrt(rx * rx + ry * ry);
  double T1, T2, T3, S1, S2;
  stress_funcs(alpha * r, T1, T2, T3, S1, S2);
  const double a2 = alpha * alpha, a4 = a2 * a2;
  const double rn = rx * nx + ry * ny;
  const double rr[2] = {rx, ry}, nn[2] = {nx, ny};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      D[2 * a + b] = -a2 * T1 * (nn[a] * rr[b] + nn[b] * rr[a] + (a == b ? rn : 0.0)) - a4 * T2 * rr[a] * rr[b] * rn -
                     a2 * T3 * rr[a] * nn[b];
}


// The double-layer kernel split by channel (the far-field bases of Sec. 3.2.1, Eqs. mpole, loc):
// every term of T1, T2, T3 either carries K0(z), K1(z) -- it comes from derivatives of
// K0(alpha r) and solves (alpha^2 - Laplacian) v = 0 away from the source (channel K) -- or is
// algebraic in r -- derivatives of log r, harmonic (channel L). DK + DL = dl_kernel. r > 0.
__device__ inline void dl_kernel_split(double alpha, double rx, double ry, double nx, double ny, double DK[4],
                                       double DL[4]) {
  const double r = sqrt(rx * rx + ry * ry);
  const double z = alpha * r;
  double k0s, k1s;
  bessel_k01_scaled(z, k0s, k1s);
  const double e = (z < 700.0) ? exp(-z) : 0.0;
  const double K0 = k0s * e, K1 = k1s * e;
  const double z2 = z * z, z4 = z2 * z2;
  const double T1K = -(2.0 * z2 * K0 + (z2 + 4.0) * z * K1) / (2.0 * kPi * z4);
  const double T2K = (4.0 * z2 * K0 + (z2 + 8.0) * z * K1) / (kPi * z4 * z2);
  const double T3K = z * K1 / (2.0 * kPi * z2);
  const double T1L = 2.0 / (kPi * z4);
  const double T2L = -8.0 / (kPi * z4 * z2);
  const double T3L = -1.0 / (2.0 * kPi * z2);
  const double a2 = alpha * alpha, a4 = a2 * a2;
  const double rn = rx * nx + ry * ny;
  const double rr[2] = {rx, ry}, nn[2] = {nx, ny};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const double sym = nn[a] * rr[b] + nn[b] * rr[a] + (a == b ? rn : 0.0);
      const double rrn = rr[a] * rr[b] * rn, rnb = rr[a] * nn[b];
      DK[2 * a + b] = -a2 * T1K * sym - a4 * T2K * rrn - a2 * T3K * rnb;
      DL[2 * a + b] = -a2 * T1L * sym - a4 * T2L * rrn - a2 * T3L * rnb;
    }
}

}  // namespace vp
