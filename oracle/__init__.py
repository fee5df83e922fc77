"""FP64 CPU oracle for the VIE path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library.  Every function follows the passage of arXiv 1610.00835 cited in
``vie_oracle.c``; this module only marshals numpy arrays through ctypes and
adds two dense helpers built on library primitives (numpy LU solve).

Parity status: all functions are pinned by the CPU tests, except
``do_solve`` (discrete-ordinates brute force), which agrees with the VIE to
discretisation level only -- parity unpinned at tight tolerance.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

TAU_MARCH, TAU_CLOSED, TAU_EXACT = 0, 1, 2
DISC_MII = 16   # or'ed into `mode`: approach M-ii (2D) instead of M-iii
OP_K_SIGMA_S, OP_I_MINUS_K, OP_A_RAW = 0, 1, 2

_lib = None
_dp = C.POINTER(C.c_double)
_lp = C.POINTER(C.c_long)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_interp.restype = C.c_double
        L.or_interp.argtypes = [C.c_int, C.c_int, _dp, _dp]
        L.or_tau_march.restype = C.c_double
        L.or_tau_march.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, C.c_int]
        L.or_tau_exact.restype = C.c_double
        L.or_tau_exact.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp]
        L.or_cell_integral2.restype = C.c_double
        L.or_cell_integral2.argtypes = [C.c_double, C.c_double, C.c_double]
        L.or_selfcell.restype = C.c_double
        L.or_selfcell.argtypes = [C.c_int, C.c_double, C.c_double]
        L.or_entry.restype = C.c_double
        L.or_entry.argtypes = [C.c_int, C.c_int, _dp, C.c_int, C.c_int, C.c_long, C.c_long]
        L.or_selfcells.restype = None
        L.or_selfcells.argtypes = [C.c_int, C.c_int, _dp, _dp]
        L.or_assemble.restype = None
        L.or_assemble.argtypes = [C.c_int, C.c_int, _dp, C.c_int, C.c_int, _dp]
        L.or_apply.restype = None
        L.or_apply.argtypes = [C.c_int, C.c_int, _dp, _dp, C.c_int, C.c_int, C.c_int,
                               _dp, _dp, _lp, C.c_long, _dp]
        L.or_gmres.restype = C.c_int
        L.or_gmres.argtypes = [C.c_int, C.c_int, _dp, _dp, C.c_int, C.c_int, _dp, _dp, _dp,
                               C.c_double, C.c_int, C.c_int, C.POINTER(C.c_int), _dp]
        L.or_exit_length.restype = C.c_double
        L.or_exit_length.argtypes = [C.c_int, _dp, _dp]
        L.or_sweep_steps.restype = C.c_long
        L.or_sweep_steps.argtypes = [C.c_int, C.c_double]
        L.or_sweep.restype = None
        L.or_sweep.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, C.c_int, _dp]
        L.or_do_solve.restype = C.c_int
        L.or_do_solve.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp, C.c_int, C.c_double,
                                  C.c_int, _dp]
        L.or_num_threads.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def num_threads() -> int:
    return lib().or_num_threads()


def set_threads(t: int) -> None:
    lib().or_set_threads(int(t))


def dim_n(sigma: np.ndarray, dim: int) -> int:
    n = int(round(sigma.size ** (1.0 / dim)))
    if n ** dim != sigma.size:
        raise ValueError("field size is not n^dim")
    return n


def interp(dim, sigma, p):
    s, sp = _d(sigma)
    q, qp = _d(p)
    return lib().or_interp(dim, dim_n(s, dim), sp, qp)


def tau_march(dim, sigma, x, y, S=64):
    s, sp = _d(sigma)
    a, ap = _d(x)
    b, bp = _d(y)
    return lib().or_tau_march(dim, dim_n(s, dim), sp, ap, bp, S)


def tau_exact(dim, sigma, x, y):
    s, sp = _d(sigma)
    a, ap = _d(x)
    b, bp = _d(y)
    return lib().or_tau_exact(dim, dim_n(s, dim), sp, ap, bp)


def cell_integral2(t1, t2, h):
    """int over the square of side h centred at (t1, t2) of |z|^{-1} dz (2D)."""
    return lib().or_cell_integral2(float(t1), float(t2), float(h))


def selfcell(dim, h, sigma):
    return lib().or_selfcell(dim, float(h), float(sigma))


def selfcells(dim, sigma_t):
    s, sp = _d(sigma_t)
    out = np.empty_like(s)
    lib().or_selfcells(dim, dim_n(s, dim), sp, out.ctypes.data_as(_dp))
    return out


def entry(dim, sigma_t, j, k, mode=TAU_MARCH, S=64):
    s, sp = _d(sigma_t)
    return lib().or_entry(dim, dim_n(s, dim), sp, mode, S, int(j), int(k))


def assemble(dim, sigma_t, mode=TAU_MARCH, S=64):
    """Dense A (N x N): off-diagonal M-iii weights and self-cell diagonal, or
    every entry by M-ii when ``mode`` carries DISC_MII."""
    s, sp = _d(sigma_t)
    N = s.size
    A = np.empty((N, N), dtype=np.float64)
    lib().or_assemble(dim, dim_n(s, dim), sp, mode, S, A.ctypes.data_as(_dp))
    return A


def apply(dim, sigma_t, sigma_s, g, op=OP_K_SIGMA_S, mode=TAU_MARCH, S=64, rows=None,
          diag=None):
    """Matrix-free apply on all rows or on the target rows ``rows``."""
    st, stp = _d(sigma_t)
    ss, ssp = _d(sigma_s)
    gg, gp = _d(g)
    n = dim_n(st, dim)
    if rows is None:
        out = np.empty(st.size)
        rp, nr = None, st.size
    else:
        r = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.empty(r.size)
        rp, nr = r.ctypes.data_as(_lp), r.size
    if diag is not None:
        dd, dp = _d(diag)
    else:
        dd, dp = None, None
    lib().or_apply(dim, n, stp, ssp, mode, S, op, dp, gp, rp, nr, out.ctypes.data_as(_dp))
    return out


def gmres(dim, sigma_t, sigma_s, phi, rtol=1e-10, restart=64, maxit=1000, mode=TAU_MARCH,
          S=64, dense=None, x0=None):
    """Restarted GMRES for (I - K) U = phi; returns (U, iters, relres, converged)."""
    st, stp = _d(sigma_t)
    ss, ssp = _d(sigma_s)
    ph, php = _d(phi)
    U = np.zeros(st.size) if x0 is None else np.array(x0, dtype=np.float64)
    if dense is not None:
        D, Dp = _d(dense)
    else:
        D, Dp = None, None
    it = C.c_int(0)
    rr = C.c_double(0.0)
    rc = lib().or_gmres(dim, dim_n(st, dim), stp, ssp, mode, S, Dp, php,
                        U.ctypes.data_as(_dp), rtol, restart, maxit, C.byref(it), C.byref(rr))
    return U, it.value, rr.value, rc == 0


def k_matrix(dim, sigma_t, sigma_s, mode=TAU_MARCH, S=64):
    """Dense K = A diag(sigma_s)."""
    return assemble(dim, sigma_t, mode, S) * np.asarray(sigma_s)[None, :]


def lu_solve(dim, sigma_t, sigma_s, phi, mode=TAU_MARCH, S=64):
    """U = (I - K)^{-1} phi by LU with partial pivoting (numpy/LAPACK)."""
    K = k_matrix(dim, sigma_t, sigma_s, mode, S)
    return np.linalg.solve(np.eye(K.shape[0]) - K, np.asarray(phi, dtype=np.float64))


def exit_length(dim, x, v):
    a, ap = _d(x)
    b, bp = _d(v)
    return lib().or_exit_length(dim, ap, bp)


def sweep_steps(n, L):
    return lib().or_sweep_steps(int(n), float(L))


def sweep(dim, sigma_t, Q, dirs):
    """Phi[m, j] for the backward characteristic from x_j along -dirs[m]."""
    st, stp = _d(sigma_t)
    q, qp = _d(Q)
    dv, dvp = _d(dirs)
    M = dv.shape[0]
    out = np.empty((M, st.size))
    lib().or_sweep(dim, dim_n(st, dim), stp, qp, dvp, M, out.ctypes.data_as(_dp))
    return out


def do_solve(dim, sigma_t, sigma_s, f, dirs, tol=1e-12, maxit=2000):
    st, stp = _d(sigma_t)
    ss, ssp = _d(sigma_s)
    ff, fp = _d(f)
    dv, dvp = _d(dirs)
    U = np.empty(st.size)
    it = lib().or_do_solve(dim, dim_n(st, dim), stp, ssp, fp, dvp, dv.shape[0], tol, maxit,
                           U.ctypes.data_as(_dp))
    return U, it
