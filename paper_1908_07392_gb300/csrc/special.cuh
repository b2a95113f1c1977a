// FP64 modified Bessel functions for the table and operator builders.
//
//  * K0, K1 for small argument (z <= 2): the power series of the paper's
//    Appendix C (I0, I1, K0, K1 with the digamma recursion psi(n+1) = psi(n)+1/n).
//  * 2 < z <= 25: the integral representation K_nu(z) = int_0^inf exp(-z cosh t)
//    cosh(nu t) dt (DLMF 10.32.9) with the trapezoidal rule, whose error decays
//    like exp(-2 pi a / h) for an integrand analytic in |Im t| < a; the step is
//    shrunk like z^-1/2 because the integrand grows like exp(z (1 - cos a)) off
//    the real axis.
//  * z > 25: the Hankel asymptotic expansion (DLMF 10.40.2), whose smallest term
//    is below exp(-2z).
//  All return exponentially scaled values e^z K_nu(z).
//
//  Normalised sequences for the expansions (no overflow for the orders and
//  arguments the FMM uses):
//    Khat_n(z) = K_n(z) (z/2)^n 2/(n-1)!   (n >= 1),  Khat_0 = K_0
//        forward recurrence with positive terms derived from
//        K_{n+1} = K_{n-1} + (2n/z) K_n (DLMF 10.29.1):
//        Khat_{n+1} = Khat_n + Khat_{n-1} z^2 / (4 n (n-1))   (n >= 2),
//        Khat_2 = Khat_1 + (z^2/2) Khat_0,   Khat_1 = z K_1.
//    Ihat_n(z) = I_n(z) n! / (z/2)^n = sum_k (z^2/4)^k n! / (k! (n+k)!)
//        (DLMF 10.25.2), positive series for the two highest orders, then the
//        backward recurrence with positive terms from I_{n-1} = I_{n+1} + (2n/z) I_n:
//        Ihat_{n-1} = Ihat_n + Ihat_{n+1} z^2 / (4 n (n+1)).
#pragma once

#include <cuda_runtime.h>

namespace vp {

constexpr double kPi = 3.14159265358979323846;
constexpr double kEulerGamma = 0.57721566490153286061;

// e^z K0(z), e^z K1(z) for z > 0.
__device__ inline void bessel_k01_scaled(double z, double& k0s, double& k1s) {
  if (z <= 2.0) {
    const double t = 0.25 * z * z;
    const double lz = log(0.5 * z);
    double i0 = 0.0, i1 = 0.0, s0 = 0.0, s1 = 0.0;
    double term0 = 1.0, term1 = 1.0, psi1 = -kEulerGamma;
    for (int n = 0; n < 20; ++n) {
      const double psi2 = psi1 + 1.0 / (n + 1);
      i0 += term0;
      i1 += term1;
      s0 += psi1 * term0;
      s1 += (psi1 + psi2) * term1;
      term0 *= t / ((n + 1.0) * (n + 1.0));
      term1 *= t / ((n + 1.0) * (n + 2.0));
      psi1 = psi2;
    }
    const double I1 = 0.5 * z * i1;
    const double K0 = -lz * i0 + s0;
    const double K1 = 1.0 / z + lz * I1 - 0.25 * z * s1;
    const double ez = exp(z);
    k0s = K0 * ez;
    k1s = K1 * ez;
  } else if (z <= 25.0) {
    const double h = fmin(0.2, 0.4 / sqrt(z));
    const double T = acosh(1.0 + 45.0 / z);
    const int n = (int)ceil(T / h);
    double a = 0.5, b = 0.5;  // t = 0 term: exp(0) * {1, cosh 0}
    for (int k = 1; k <= n; ++k) {
      const double t = k * h;
      const double c = cosh(t);
      const double g = exp(-z * (c - 1.0));
      a += g;
      b += g * c;
    }
    k0s = h * a;
    k1s = h * b;
  } else {
    const double pre = sqrt(0.5 * kPi / z);
    double out[2];
    for (int nu = 0; nu < 2; ++nu) {
      const double mu = 4.0 * nu * nu;
      double s = 1.0, term = 1.0;
      for (int k = 1; k < 40; ++k) {
        const double f = (2.0 * k - 1.0);
        term *= (mu - f * f) / (8.0 * k * z);
        s += term;
        if (fabs(term) < 1e-17 * fabs(s)) break;
      }
      out[nu] = pre * s;
    }
    k0s = out[0];
    k1s = out[1];
  }
}

// e^z * Khat_n(z), n = 0..nmax (nmax >= 1).
__device__ inline void khat_scaled(double z, int nmax, double* kh) {
  double k0s, k1s;
  bessel_k01_scaled(z, k0s, k1s);
  kh[0] = k0s;
  kh[1] = z * k1s;
  if (nmax >= 2) kh[2] = kh[1] + 0.5 * z * z * k0s;
  for (int n = 2; n < nmax; ++n) kh[n + 1] = kh[n] + kh[n - 1] * z * z / (4.0 * n * (n - 1.0));
}

__device__ inline double ihat_series(double z, int n) {
  const double t = 0.25 * z * z;
  double s = 0.0, term = 1.0;
  for (int k = 1; k < 400; ++k) {
    s += term;
    term *= t / (k * (double)(n + k));
    if (term < 1e-17 * s) break;
  }
  return s + term;
}

// Ihat_n(z), n = 0..nmax.
__device__ inline void ihat(double z, int nmax, double* ih) {
  ih[nmax] = ihat_series(z, nmax);
  if (nmax == 0) return;
  ih[nmax - 1] = ihat_series(z, nmax - 1);
  for (int n = nmax - 1; n >= 1; --n) ih[n - 1] = ih[n] + ih[n + 1] * z * z / (4.0 * n * (n + 1.0));
}

// G, dG/dx, dG/dy at displacement (dx, dy) = x - y for the full kernel.
//   kernel 0: G1 = K0(a r)/(2 pi); kernel 1: G2 = (K0(a r) + log r)/(2 pi a^2).
__device__ inline void kernel_full(int kernel, double alpha, double dx, double dy, double& g,
                                   double& gx, double& gy) {
  const double r = sqrt(dx * dx + dy * dy);
  const double z = alpha * r;
  double k0 = 0.0, k1 = 0.0;
  if (z < 700.0) {
    double k0s, k1s;
    bessel_k01_scaled(z, k0s, k1s);
    const double e = exp(-z);
    k0 = k0s * e;
    k1 = k1s * e;
  }
  double gp;
  if (kernel == 0) {
    g = k0 * (0.5 / kPi);
    gp = -alpha * k1 * (0.5 / kPi);
  } else {
    const double s = 0.5 / (kPi * alpha * alpha);
    g = (k0 + log(r)) * s;
    gp = (1.0 / r - alpha * k1) * s;
  }
  gx = gp * dx / r;
  gy = gp * dy / r;
}

}  // namespace vp
