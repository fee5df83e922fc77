"""Pins of the oracle's interpolation-based FMM (Section 3.3): its march
against the pinned C march, the Chebyshev interpolation against polynomials,
the tree's near and far lists against an exact cover of all leaf pairs, and
the FMM apply against the direct apply (spectral in the order p for a
homogeneous medium, as in Table TAB:Con Coeff)."""
import numpy as np
import pytest

import oracle as O
import vie_synth as V
from oracle import fmm as F


def test_vectorised_march_equals_the_oracle_march():
    n = 17
    m = V.bump_medium(2, n, 4, 0.9, seed=81)
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, (40, 2))
    y = rng.uniform(0, 1, (40, 2))
    x[:5] = [[0.0, 0.0], [1.0, 1.0], [0.01, 0.99], [0.5, 0.0], [0.999, 0.3]]   # outside the centre hull
    want = np.array([O.tau_march(2, m.sigma_t, a, b) for a, b in zip(x, y)])
    np.testing.assert_allclose(F.tau_march(m.sigma_t, n, x, y), want, rtol=1e-13, atol=0)


@pytest.mark.parametrize("p", [3, 6, 9])
def test_chebyshev_interpolation_reproduces_polynomials(p):
    # sum_m S_p(u, z_m) q(z_m) = q(u) for every polynomial of degree < p per axis
    rng = np.random.default_rng(p)
    c = rng.standard_normal((p, p))
    q = lambda x, y: np.polynomial.polynomial.polyval2d(x, y, c)  # noqa: E731
    nodes = F.box_nodes(p, (0.25, 0.5), 0.125)
    pts = np.column_stack([rng.uniform(0.25, 0.375, 30), rng.uniform(0.5, 0.625, 30)])
    M = F.interp_matrix(p, pts, (0.25, 0.5), 0.125)       # [p^2, k]
    np.testing.assert_allclose(M.T @ q(nodes[:, 0], nodes[:, 1]), q(pts[:, 0], pts[:, 1]), rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("n", [32, 64, 96])
def test_near_and_far_lists_cover_every_leaf_pair_once(n):
    L, b = F.leaf_levels(n)
    nl = 2 ** L
    count = {}
    for by in range(nl):
        for bx in range(nl):
            for cy in range(nl):
                for cx in range(nl):
                    if abs(bx - cx) <= 1 and abs(by - cy) <= 1:
                        count[(bx, by, cx, cy)] = count.get((bx, by, cx, cy), 0) + 1
    for lev in range(2, L + 1):
        nb, sh = 2 ** lev, L - lev
        for by in range(nb):
            for bx in range(nb):
                for (cx, cy) in F.interaction_list(lev, (bx, by)):
                    for ty in range(by << sh, (by + 1) << sh):
                        for tx in range(bx << sh, (bx + 1) << sh):
                            for sy in range(cy << sh, (cy + 1) << sh):
                                for sx in range(cx << sh, (cx + 1) << sh):
                                    count[(tx, ty, sx, sy)] = count.get((tx, ty, sx, sy), 0) + 1
    assert len(count) == nl ** 4 and set(count.values()) == {1}


def test_fmm_converges_spectrally_on_a_homogeneous_medium():
    n = 32
    st = np.full(n * n, 2.2)
    g = np.random.default_rng(5).standard_normal(n * n)
    want = O.apply(2, st, st, g, op=O.OP_A_RAW)
    errs = [np.linalg.norm(F.apply(st, g, n, p) - want) / np.linalg.norm(want) for p in (4, 7, 10)]
    assert errs[0] > 30 * errs[1] > 30 * 30 * errs[2]
    assert errs[2] < 1e-8


def test_fmm_on_a_heterogeneous_medium():
    # the kernel's exp(-tau) of a bilinear sigma_t is only piecewise smooth:
    # the error levels off near 1e-5 .. 1e-4 (Table TAB:Var Coeff: 2e-4 .. 4e-4 at order 4)
    n = 32
    m = V.bump_medium(2, n, 4, 0.9, seed=82)
    g = np.random.default_rng(6).standard_normal(n * n)
    want = O.apply(2, m.sigma_t, m.sigma_s, g, op=O.OP_A_RAW)
    assert np.linalg.norm(F.apply(m.sigma_t, g, n, 6) - want) / np.linalg.norm(want) < 2e-4
