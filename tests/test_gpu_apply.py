"""Parity of the CUDA operator apply with the FP64 oracle (element by element)."""
import numpy as np
import pytest

import oracle as O
import vie_synth as V

torch = pytest.importorskip("torch")
import paper_1610_00835_gb300 as P  # noqa: E402
from gpu_util import dev, host, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5   # relative L2 bar for FP32 kernel tiles
FP64_TOL = 1e-12


def gpu_apply(h, op, g, nrhs=1):
    y = torch.empty(nrhs * h.N, dtype=torch.float64, device="cuda:0")
    P.vie_apply(h, op, dev(g), y, nrhs)
    return host(y)


def rng_vec(N, seed=0):
    return np.random.default_rng(seed).standard_normal(N)


def test_homogeneous_fp64_closed_form_config1():
    m = V.homogeneous_medium(2, 32, 1.1, 1.0)
    h = P.vie_create(2, 32, m.sigma_t, m.sigma_s, tau_mode=P.VIE_TAU_CLOSED,
                     precision=P.VIE_PREC_FP64)
    for op in (P.VIE_OP_K_SIGMA_S, P.VIE_OP_A_RAW, P.VIE_OP_I_MINUS_K):
        g = rng_vec(m.N, op)
        want = O.apply(2, m.sigma_t, m.sigma_s, g, op=op, mode=O.TAU_CLOSED)
        assert rel_l2(gpu_apply(h, op, g), want) < FP64_TOL


@pytest.mark.parametrize("n", [1, 2, 3, 17, 24, 40])
def test_2d_fp32_march_all_rows(n):
    # several 256-target tiles plus a ragged tail; n = 1..3 are degenerate grids
    m = V.heterogeneous_2d(n=n, seed=77)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    g = rng_vec(m.N, n) + 1.0
    want = O.apply(2, m.sigma_t, m.sigma_s, g)
    got = gpu_apply(h, P.VIE_OP_K_SIGMA_S, g)
    assert rel_l2(got, want) < FP32_TOL
    assert np.max(np.abs(got - want)) < 1e-4 * np.max(np.abs(want)) + 1e-300


@pytest.mark.parametrize("n", [1, 2, 5, 10, 13])
def test_3d_fp32_march_all_rows(n):
    m = V.heterogeneous_3d(n=n, seed=88)
    h = P.vie_create(3, n, m.sigma_t, m.sigma_s)
    g = rng_vec(m.N, n) + 1.0
    want = O.apply(3, m.sigma_t, m.sigma_s, g)
    assert rel_l2(gpu_apply(h, P.VIE_OP_K_SIGMA_S, g), want) < FP32_TOL


@pytest.mark.parametrize("dim,n,S", [(2, 20, 1), (2, 20, 7), (2, 31, 100), (3, 7, 13)])
def test_runtime_step_counts(dim, n, S):
    m = V.heterogeneous_2d(n=n) if dim == 2 else V.heterogeneous_3d(n=n)
    h = P.vie_create(dim, n, m.sigma_t, m.sigma_s, steps=S)
    g = rng_vec(m.N, 3)
    want = O.apply(dim, m.sigma_t, m.sigma_s, g, S=S)
    assert rel_l2(gpu_apply(h, P.VIE_OP_K_SIGMA_S, g), want) < FP32_TOL


@pytest.mark.parametrize("dim,n", [(2, 14), (3, 6)])
def test_fp64_march_matches_oracle_to_rounding(dim, n):
    m = V.heterogeneous_2d(n=n) if dim == 2 else V.heterogeneous_3d(n=n)
    h = P.vie_create(dim, n, m.sigma_t, m.sigma_s, precision=P.VIE_PREC_FP64)
    g = rng_vec(m.N, 5)
    want = O.apply(dim, m.sigma_t, m.sigma_s, g)
    assert rel_l2(gpu_apply(h, P.VIE_OP_K_SIGMA_S, g), want) < FP64_TOL


def test_ops_and_multiple_rhs_and_host_pointers():
    n = 21
    m = V.heterogeneous_2d(n=n)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    G = np.stack([rng_vec(m.N, s) for s in range(3)])
    y_dev = gpu_apply(h, P.VIE_OP_I_MINUS_K, G.ravel(), nrhs=3).reshape(3, -1)
    y_host = np.empty(3 * m.N)
    P.vie_apply(h, P.VIE_OP_I_MINUS_K, np.ascontiguousarray(G.ravel()), y_host, 3)
    np.testing.assert_array_equal(y_dev.ravel(), y_host)
    for r in range(3):
        want = O.apply(2, m.sigma_t, m.sigma_s, G[r], op=O.OP_I_MINUS_K)
        assert rel_l2(y_dev[r], want) < FP32_TOL
    a = gpu_apply(h, P.VIE_OP_A_RAW, G[0])
    assert rel_l2(a, O.apply(2, m.sigma_t, m.sigma_s, G[0], op=O.OP_A_RAW)) < FP32_TOL


@pytest.mark.parametrize("kernel", [P.VIE_KERNEL_SYMMETRIC, P.VIE_KERNEL_DISPLACEMENT])
def test_deterministic(kernel):
    # fixed summation order (tile pairs) or exact fixed-point sums
    # (displacement kernel): repeated applies are bitwise identical
    m = V.heterogeneous_2d(n=48)
    g = rng_vec(m.N, 9)
    h = P.vie_create(2, 48, m.sigma_t, m.sigma_s, kernel=kernel)
    np.testing.assert_array_equal(gpu_apply(h, 0, g), gpu_apply(h, 0, g))


@pytest.mark.parametrize("kernel", [P.VIE_KERNEL_SYMMETRIC, P.VIE_KERNEL_DISPLACEMENT,
                                    P.VIE_KERNEL_GENERAL])
@pytest.mark.parametrize("n", [2, 3, 9, 24, 37, 64])
def test_2d_every_pair_kernel_all_rows(kernel, n):
    m = V.heterogeneous_2d(n=n, seed=78)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s, kernel=kernel)
    g = rng_vec(m.N, n) + 0.5
    for op in (P.VIE_OP_K_SIGMA_S, P.VIE_OP_A_RAW):
        want = O.apply(2, m.sigma_t, m.sigma_s, g, op=op)
        assert rel_l2(gpu_apply(h, op, g), want) < FP32_TOL


@pytest.mark.parametrize("n", [100, 128, 133, 226, 233, 234, 256, 258])
def test_displacement_kernel_full_size_sampled_rows(n):
    # 233 is the largest grid whose lattice ((n + 8) rows of an odd pitch) fits
    # one SM's shared memory; 234 ... 258 read it from global memory (two
    # layouts, runs along y and x)
    m = V.bump_medium(2, n, 4, 0.9, seed=4300 + n)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s, kernel=P.VIE_KERNEL_DISPLACEMENT)
    assert P.vie_get_kernel(h) == P.VIE_KERNEL_DISPLACEMENT
    hs = P.vie_create(2, n, m.sigma_t, m.sigma_s, kernel=P.VIE_KERNEL_SYMMETRIC)
    g = m.f + 0.05 * rng_vec(m.N, n)
    got = gpu_apply(h, P.VIE_OP_K_SIGMA_S, g)
    rows = _sampled_rows(m.N, 16, n)
    want = O.apply(2, m.sigma_t, m.sigma_s, g, rows=rows)
    assert rel_l2(got[rows], want) < FP32_TOL
    assert rel_l2(got, gpu_apply(hs, P.VIE_OP_K_SIGMA_S, g)) < 2e-6


def test_displacement_kernel_falls_back_beyond_its_lattice():
    # n = 259 is past the global lattice (267 x 267 with the stacked-target
    # padding): the handle takes the tile-pair kernel and still matches the oracle
    n = 259
    m = V.bump_medium(2, n, 4, 0.9, seed=4436)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s, kernel=P.VIE_KERNEL_DISPLACEMENT)
    assert P.vie_get_kernel(h) == P.VIE_KERNEL_SYMMETRIC
    g = m.f + 0.05 * rng_vec(m.N, n)
    rows = _sampled_rows(m.N, 8, n)
    want = O.apply(2, m.sigma_t, m.sigma_s, g, rows=rows)
    assert rel_l2(gpu_apply(h, P.VIE_OP_K_SIGMA_S, g)[rows], want) < FP32_TOL


@pytest.mark.parametrize("dim,n", [(2, 9), (3, 5)])
def test_selfcell_diagonal(dim, n):
    m = V.heterogeneous_2d(n=n) if dim == 2 else V.heterogeneous_3d(n=n)
    h = P.vie_create(dim, n, m.sigma_t, m.sigma_s)
    d = np.empty(m.N)
    P.vie_get_diagonal(h, d)
    np.testing.assert_allclose(d, O.selfcells(dim, m.sigma_t), rtol=1e-12)


def test_reciprocity_on_gpu():
    # columns of A from unit vectors: A_jk = A_kj up to FP32 rounding
    n = 8
    m = V.heterogeneous_2d(n=n)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    A = gpu_apply(h, P.VIE_OP_A_RAW, np.eye(m.N).ravel(), nrhs=m.N).reshape(m.N, m.N).T
    off = ~np.eye(m.N, dtype=bool)
    assert np.max(np.abs(A - A.T)[off] / A[off]) < 2e-6


def _sampled_rows(N, count, seed):
    r = np.random.default_rng(seed).choice(N, size=count, replace=False)
    return np.unique(np.concatenate([r, [0, N - 1, N // 2]]))


def test_config2_full_size_sampled_rows():
    m = V.heterogeneous_2d()
    h = P.vie_create(2, m.n, m.sigma_t, m.sigma_s)
    g = m.f + 0.1 * rng_vec(m.N, 11)
    got = gpu_apply(h, P.VIE_OP_K_SIGMA_S, g)
    rows = _sampled_rows(m.N, 40, 1)
    want = O.apply(2, m.sigma_t, m.sigma_s, g, rows=rows)
    assert rel_l2(got[rows], want) < FP32_TOL


@pytest.mark.parametrize("n", [2, 3, 8, 32])
def test_3d_displacement_kernel_against_tile_pairs_and_oracle(n):
    # 3D grids up to 32^3 take the displacement kernel; it agrees with the
    # tile-pair kernel, the oracle (sampled rows) and itself (bitwise)
    m = V.heterogeneous_3d(n=n, seed=90 + n)
    h = P.vie_create(3, n, m.sigma_t, m.sigma_s)
    assert P.vie_get_kernel(h) == P.VIE_KERNEL_DISPLACEMENT
    hs = P.vie_create(3, n, m.sigma_t, m.sigma_s, kernel=P.VIE_KERNEL_SYMMETRIC)
    assert P.vie_get_kernel(hs) == P.VIE_KERNEL_SYMMETRIC
    g = m.f + 0.1 * rng_vec(m.N, n)
    for op in (P.VIE_OP_K_SIGMA_S, P.VIE_OP_A_RAW, P.VIE_OP_I_MINUS_K):
        got = gpu_apply(h, op, g)
        assert rel_l2(got, gpu_apply(hs, op, g)) < 2e-6
        np.testing.assert_array_equal(gpu_apply(h, op, g), got)
    rows = _sampled_rows(m.N, min(12, m.N), n + 3)
    want = O.apply(3, m.sigma_t, m.sigma_s, g, rows=rows)
    assert rel_l2(gpu_apply(h, P.VIE_OP_K_SIGMA_S, g)[rows], want) < FP32_TOL


def test_3d_beyond_32_takes_another_kernel():
    m = V.heterogeneous_3d(n=33, seed=97)
    h = P.vie_create(3, 33, m.sigma_t, m.sigma_s)
    assert P.vie_get_kernel(h) != P.VIE_KERNEL_DISPLACEMENT
    g = m.f
    rows = _sampled_rows(m.N, 6, 33)
    want = O.apply(3, m.sigma_t, m.sigma_s, g, rows=rows)
    assert rel_l2(gpu_apply(h, P.VIE_OP_K_SIGMA_S, g)[rows], want) < FP32_TOL


def test_config3_full_size_sampled_rows():
    m = V.heterogeneous_3d()
    h = P.vie_create(3, m.n, m.sigma_t, m.sigma_s)
    g = m.f + 0.1 * rng_vec(m.N, 12)
    got = gpu_apply(h, P.VIE_OP_K_SIGMA_S, g)
    rows = _sampled_rows(m.N, 24, 2)
    want = O.apply(3, m.sigma_t, m.sigma_s, g, rows=rows)
    assert rel_l2(got[rows], want) < FP32_TOL


def test_256_grid_global_sigma_path_sampled_rows():
    # sigma_t of a 256^2 grid does not fit in shared memory: global-load path
    m = V.bump_medium(2, 256, 4, 0.9, seed=4015)
    h = P.vie_create(2, 256, m.sigma_t, m.sigma_s)
    g = m.f
    got = gpu_apply(h, P.VIE_OP_K_SIGMA_S, g)
    rows = _sampled_rows(m.N, 8, 3)
    want = O.apply(2, m.sigma_t, m.sigma_s, g, rows=rows)
    assert rel_l2(got[rows], want) < FP32_TOL


@pytest.mark.parametrize("n", [31, 33, 64, 65, 96, 150, 200, 224])
def test_symmetric_kernel_every_lattice_stride(n):
    # the symmetric FP32 kernel is compiled for lattice strides 33..225; each
    # size here lands in a different one, with a ragged last tile
    m = V.bump_medium(2, n, 4, 0.9, seed=4100 + n)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    g = m.f + 0.05 * rng_vec(m.N, n)
    got = gpu_apply(h, P.VIE_OP_K_SIGMA_S, g)
    rows = _sampled_rows(m.N, 16, n)
    want = O.apply(2, m.sigma_t, m.sigma_s, g, rows=rows)
    assert rel_l2(got[rows], want) < FP32_TOL


def test_handles_of_different_sizes_share_kernel_instances():
    # grids 40 and 23 run the same displacement-kernel instance with different
    # shared-memory sizes; creating the smaller one must not break the larger
    media = {n: V.bump_medium(2, n, 3, 0.9, seed=4950 + n) for n in (40, 23, 100)}
    handles = {n: P.vie_create(2, n, m.sigma_t, m.sigma_s) for n, m in media.items()}
    for n, h in handles.items():
        assert P.vie_get_kernel(h) == P.VIE_KERNEL_DISPLACEMENT
        m = media[n]
        g = m.f + 0.05 * rng_vec(m.N, n)
        rows = _sampled_rows(m.N, 6, n)
        want = O.apply(2, m.sigma_t, m.sigma_s, g, rows=rows)
        assert rel_l2(gpu_apply(h, P.VIE_OP_K_SIGMA_S, g)[rows], want) < FP32_TOL
