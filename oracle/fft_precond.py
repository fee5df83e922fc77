"""FFT preconditioner of Section 4.4 (Eqs. EQ: FFT and EQ:SOL FFT), FP64 numpy
reference (TEST INFRASTRUCTURE ONLY: imported by tests/ and nothing else).

The preconditioner replaces sigma_t and sigma_s by their means over the grid,
mu = mean sigma_t and mu_s = mean sigma_s.  With constant coefficients the
discrete operator is a convolution, U - mu_s W * U = b, whose kernel W is the
matrix A of a homogeneous medium, a function of the displacement only:
    M-iii: W(D) = h^2 exp(-mu h|D|) / (2 pi h|D|) for D != 0,
           W(0) = the self-cell integral with sigma frozen at mu;
    M-ii : W(D) = exp(-mu h|D|) / (2 pi) int_{T(hD)} |z|^{-1} dz (W(0) with tau = 0).
The convolution is extended periodically to a square of m >= 2n cells per side
(the paper's [0, 2]^d, here rounded up to a power of two), the vector is
extended by zero (the paper's regularisation P^{-1} g = g chi_Omega), the
periodic operator is inverted by the discrete Fourier transform, and the
result restricted to the grid:
    z = P F^{-1}( F(P^{-1} b) / F(delta - mu_s W~) ).
The DFT is numpy's (a library primitive).  2D only.
"""
from __future__ import annotations

import numpy as np

from . import cell_integral2, selfcell


def grid_size(n: int) -> int:
    """Side m of the periodic square: the smallest power of two >= 2 n."""
    m = 1
    while m < 2 * n:
        m *= 2
    return m


def kernel_on_torus(n: int, mu: float, m: int, mii: bool = False) -> np.ndarray:
    """W~[iy, ix]: W at the displacement (dx, dy) = (ix, iy) taken in [-m/2, m/2)."""
    h = 1.0 / n
    d = np.arange(m)
    d = np.where(d < m // 2, d, d - m)
    W = np.empty((m, m))
    for iy in range(m):
        for ix in range(m):
            dx, dy = d[ix], d[iy]
            r = h * np.hypot(dx, dy)
            if mii:
                W[iy, ix] = np.exp(-mu * r) * cell_integral2(dx * h, dy * h, h) / (2 * np.pi)
            elif dx == 0 and dy == 0:
                W[iy, ix] = selfcell(2, h, mu)
            else:
                W[iy, ix] = h * h * np.exp(-mu * r) / (2 * np.pi * r)
    return W


def symbol(n: int, mu: float, mu_s: float, mii: bool = False) -> np.ndarray:
    """F(delta - mu_s W~): the eigenvalues of the periodic operator."""
    m = grid_size(n)
    return 1.0 - mu_s * np.fft.fft2(kernel_on_torus(n, mu, m, mii))


def precondition(b, n: int, mu: float, mu_s: float, mii: bool = False) -> np.ndarray:
    """z = P F^{-1}(F(P^{-1} b) / F(delta - mu_s W~)) for b on the n x n grid."""
    m = grid_size(n)
    B = np.zeros((m, m))
    B[:n, :n] = np.asarray(b, dtype=np.float64).reshape(n, n)
    Z = np.fft.ifft2(np.fft.fft2(B) / symbol(n, mu, mu_s, mii))
    return Z.real[:n, :n].ravel()


def precondition_medium(b, sigma_t, sigma_s, n: int, mii: bool = False) -> np.ndarray:
    """The preconditioner of a medium: its coefficients replaced by their means."""
    return precondition(b, n, float(np.mean(sigma_t)), float(np.mean(sigma_s)), mii)
