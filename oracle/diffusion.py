"""Diffusion preconditioner of Section 4.4 (Eq. EQ:DA), FP64 numpy/scipy
reference (TEST INFRASTRUCTURE ONLY: imported by tests/ and nothing else).

Diffusion approximation on the unit square (d = 2):
    -div( kappa grad U ) + mu_a U = f,   kappa = 1 / (d mu),  mu_a = mu - mu_s,
    U + l dU/dn = 0 on the boundary,     l = 2 / (d mu),
with mu = sigma_t and mu_s = sigma_s per cell.  Second-order finite volumes on
the n x n cells (h = 1/n, index j = ix + n iy): an interior face carries the
harmonic mean of its two cells' kappa and the flux kappa_f (U_c - U_nb) / h; a
boundary face eliminates the boundary value through the Robin condition, which
leaves the outward flux 2 kappa_c U_c / (h + 2 l_c).  Divided by the cell area:
    (D U)_c = sum_interior kappa_f (U_c - U_nb) / h^2
              + sum_boundary 2 kappa_c U_c / (h (h + 2 l_c)) + mu_a,c U_c.

Preconditioner for (I - K) U = b (reading of the section: the diffusion limit
of A is (D + Sigma_s)^{-1}, so (I - A Sigma_s)^{-1} is close to
I + D^{-1} Sigma_s, the diffusion-synthetic-acceleration form on U):
    M(r) = r + D^{-1}(sigma_s r),
D^{-1} taken as V-cycles of a geometric multigrid (the section's "standard
V-cycle") from a zero guess:
    levels   : n_0 = n, n_{l+1} = n_l / 2 while n_l is even and above 8;
               coarse mu and mu_s are the means of the 2 x 2 children and the
               operator is rediscretised with h_{l+1} = 2 h_l;
    smoother : red-black Gauss-Seidel (red: ix + iy even, first), 2 sweeps
               before and 2 after the coarse correction;
    transfer : restriction = mean of the 2 x 2 children's residuals;
               prolongation = bilinear in the cell centres (weights 9/16,
               3/16, 3/16, 1/16), a neighbour outside the grid replaced by
               the coarse cell itself;
    coarsest : 200 red-black sweeps from zero.
scipy's sparse direct solve gives D^{-1} exactly for the pins.  2D only.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

PRE = POST = 2
COARSE_SWEEPS = 200


def coefficients(sigma_t, sigma_s, n):
    mu = np.asarray(sigma_t, dtype=np.float64).reshape(n, n)
    mus = np.asarray(sigma_s, dtype=np.float64).reshape(n, n)
    return mu, mu - mus


def operator(mu, mu_a):
    """The finite-volume matrix D (CSR) of the n x n grid, mu and mu_a [iy, ix]."""
    n = mu.shape[0]
    h = 1.0 / n
    kap = 1.0 / (2.0 * mu)
    ell = 2.0 / (2.0 * mu)
    rows, cols, vals = [], [], []
    for iy in range(n):
        for ix in range(n):
            c = ix + n * iy
            diag = mu_a[iy, ix]
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                jx, jy = ix + dx, iy + dy
                if 0 <= jx < n and 0 <= jy < n:
                    kf = 2.0 * kap[iy, ix] * kap[jy, jx] / (kap[iy, ix] + kap[jy, jx])
                    diag += kf / (h * h)
                    rows.append(c)
                    cols.append(jx + n * jy)
                    vals.append(-kf / (h * h))
                else:
                    diag += 2.0 * kap[iy, ix] / (h * (h + 2.0 * ell[iy, ix]))
            rows.append(c)
            cols.append(c)
            vals.append(diag)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n * n, n * n))


def solve(sigma_t, sigma_s, f, n):
    """D^{-1} f by a sparse direct solve."""
    mu, mu_a = coefficients(sigma_t, sigma_s, n)
    return spla.spsolve(operator(mu, mu_a).tocsc(), np.asarray(f, dtype=np.float64))


def hierarchy(mu, mu_a):
    """[(D_l, n_l)] from the fine grid down."""
    levels = []
    while True:
        n = mu.shape[0]
        levels.append((operator(mu, mu_a), n))
        if n % 2 or n <= 8:
            return levels
        mu = 0.25 * (mu[0::2, 0::2] + mu[1::2, 0::2] + mu[0::2, 1::2] + mu[1::2, 1::2])
        mu_a = 0.25 * (mu_a[0::2, 0::2] + mu_a[1::2, 0::2] + mu_a[0::2, 1::2] + mu_a[1::2, 1::2])


def rbgs(D, n, f, u, sweeps):
    """Red-black Gauss-Seidel sweeps (red cells first) on D u = f."""
    ix, iy = np.meshgrid(np.arange(n), np.arange(n))
    color = ((ix + iy) % 2).ravel()
    diag = D.diagonal()
    for _ in range(sweeps):
        for c in (0, 1):
            sel = color == c
            r = f - D @ u
            u[sel] += r[sel] / diag[sel]
    return u


def restrict(r, n):
    R = r.reshape(n, n)
    return (0.25 * (R[0::2, 0::2] + R[1::2, 0::2] + R[0::2, 1::2] + R[1::2, 1::2])).ravel()


def prolong(e, nc):
    """Bilinear interpolation of the coarse cell values to the fine cells."""
    E = e.reshape(nc, nc)
    n = 2 * nc
    out = np.empty((n, n))
    for fy in range(n):
        for fx in range(n):
            I, J = fx // 2, fy // 2
            sx = 1 if fx % 2 else -1
            sy = 1 if fy % 2 else -1
            I2 = I + sx if 0 <= I + sx < nc else I
            J2 = J + sy if 0 <= J + sy < nc else J
            out[fy, fx] = (9 * E[J, I] + 3 * E[J, I2] + 3 * E[J2, I] + E[J2, I2]) / 16.0
    return out.ravel()


def vcycle(levels, f, l=0):
    D, n = levels[l]
    u = np.zeros(n * n)
    if l == len(levels) - 1:
        return rbgs(D, n, f, u, COARSE_SWEEPS)
    u = rbgs(D, n, f, u, PRE)
    e = vcycle(levels, restrict(f - D @ u, n), l + 1)
    u += prolong(e, n // 2)
    return rbgs(D, n, f, u, POST)


def precondition(r, sigma_t, sigma_s, n, cycles=1):
    """M(r) = r + D^{-1}(sigma_s r), D^{-1} by `cycles` V-cycles from zero."""
    mu, mu_a = coefficients(sigma_t, sigma_s, n)
    levels = hierarchy(mu, mu_a)
    s = np.asarray(sigma_s, dtype=np.float64) * np.asarray(r, dtype=np.float64)
    e = np.zeros(n * n)
    for _ in range(cycles):
        e += vcycle(levels, s - levels[0][0] @ e)
    return np.asarray(r, dtype=np.float64) + e
