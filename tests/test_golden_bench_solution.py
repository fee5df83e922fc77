"""The stored FP64 oracle solution of the benchmark medium satisfies the
oracle's own equation (I - K) U = A f on sampled rows (Algorithm 1, S.1-S.2).
It guards the file that tests/golden/make_bench_solution.py writes."""
import json
import os

import numpy as np

import oracle as O
import vie_synth as V

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_bench_solution_residual_on_sampled_rows():
    U = np.load(os.path.join(GOLDEN, "bench_U_2d_128.npy"))
    with open(os.path.join(GOLDEN, "bench_U_2d_128.json")) as fh:
        meta = json.load(fh)
    m = V.heterogeneous_2d(n=128, seed=V.seed_for(2, 0))
    assert U.shape == (m.N,) and np.all(np.isfinite(U))
    rows = np.unique(np.concatenate([np.random.default_rng(7).choice(m.N, 6, replace=False),
                                     [0, m.N - 1, m.N // 2 + 64]]))
    diag = O.selfcells(2, m.sigma_t)
    KU = O.apply(2, m.sigma_t, m.sigma_s, U, rows=rows, diag=diag)
    phi = O.apply(2, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW, rows=rows, diag=diag)
    resid = U[rows] - KU - phi
    # |r_j| <= ||r||_2 = relres ||phi||_2 <= relres ||U||_2 (0 <= phi <= U), plus rounding
    assert np.max(np.abs(resid)) <= 2 * meta["relres"] * np.linalg.norm(U) + 1e-12 * np.max(np.abs(U))
    # U >= phi >= 0 for a non-negative source (Neumann series of a positive operator)
    assert np.all(U[rows] >= phi - 1e-12) and np.all(phi >= 0)


def test_bench_solution_mii_residual_on_sampled_rows():
    # the same check for the M-ii discretisation (Remark REM: NEW KERNEL)
    U = np.load(os.path.join(GOLDEN, "bench_U_2d_128_mii.npy"))
    with open(os.path.join(GOLDEN, "bench_U_2d_128_mii.json")) as fh:
        meta = json.load(fh)
    m = V.heterogeneous_2d(n=128, seed=V.seed_for(2, 0))
    mode = O.TAU_MARCH | O.DISC_MII
    assert U.shape == (m.N,) and np.all(np.isfinite(U))
    rows = np.unique(np.concatenate([np.random.default_rng(8).choice(m.N, 6, replace=False),
                                     [0, m.N - 1, m.N // 2 + 64]]))
    KU = O.apply(2, m.sigma_t, m.sigma_s, U, rows=rows, mode=mode)
    phi = O.apply(2, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW, rows=rows, mode=mode)
    resid = U[rows] - KU - phi
    assert np.max(np.abs(resid)) <= 2 * meta["relres"] * np.linalg.norm(U) + 1e-12 * np.max(np.abs(U))
    assert np.all(U[rows] >= phi - 1e-12) and np.all(phi >= 0)
