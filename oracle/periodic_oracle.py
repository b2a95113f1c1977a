"""Oracle of the periodic particular solution (test infrastructure only).

Sec. 2.1 (Eqs. uhat, periodic_stokeslet, uP_Fourier, uP_Fourier_deriv) written out with numpy's
FFT on the uniform n x n grid of a periodic box of side L: F_hat = FFT(F), u_hat = S_hat F_hat with
S_hat(k) = (I - k k^T / |k|^2) / (alpha^2 + |k|^2) and S_hat(0) = I / alpha^2, u = IFFT(u_hat),
grad u = IFFT(i k u_hat) (wavenumber n/2, the Nyquist mode, differentiates to zero on the grid).
Arrays are [component][row j (y)][column i (x)]. Nothing here is shared with the CUDA path.
"""
from __future__ import annotations

import numpy as np


def wavenumbers(n, L):
    k = 2 * np.pi / L * np.fft.fftfreq(n, d=1.0 / n)
    kd = k.copy()
    kd[n // 2] = 0.0  # Nyquist: no derivative
    return k, kd


def periodic_stokes(alpha, L, F):
    F = np.asarray(F, float)
    n = F.shape[-1]
    k, kd = wavenumbers(n, L)
    KY, KX = np.meshgrid(k, k, indexing="ij")
    DY, DX = np.meshgrid(kd, kd, indexing="ij")
    K2 = KX ** 2 + KY ** 2
    Fh = np.fft.fft2(F, axes=(-2, -1))
    with np.errstate(divide="ignore", invalid="ignore"):
        den = np.where(K2 > 0, 1.0 / (K2 * (alpha ** 2 + K2)), 0.0)
    S = np.empty((2, 2) + K2.shape)
    S[0, 0] = np.where(K2 > 0, KY ** 2 * den, 1.0 / alpha ** 2)
    S[1, 1] = np.where(K2 > 0, KX ** 2 * den, 1.0 / alpha ** 2)
    S[0, 1] = S[1, 0] = np.where(K2 > 0, -KX * KY * den, 0.0)
    uh = np.einsum("ab...,b...->a...", S, Fh)
    u = np.real(np.fft.ifft2(uh, axes=(-2, -1)))
    g = np.empty((2, 2) + K2.shape)
    for a in range(2):
        g[a, 0] = np.real(np.fft.ifft2(1j * DX * uh[a]))
        g[a, 1] = np.real(np.fft.ifft2(1j * DY * uh[a]))
    return u, g
