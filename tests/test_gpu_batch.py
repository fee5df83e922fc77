"""One persistent launch over uneven 2D grids (CUDA graph, autotuned) vs the oracle."""
import os

import numpy as np
import pytest

import oracle as O
import vie_synth as V

torch = pytest.importorskip("torch")
import paper_1610_00835_gb300 as P  # noqa: E402
from gpu_util import dev, host, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-5


def make_batch(ns, seed0=300, kernel=P.VIE_KERNEL_AUTO):
    media = [V.bump_medium(2, n, 4, 0.9, seed=seed0 + i) for i, n in enumerate(ns)]
    b = P.vie_batch_create(ns, [m.sigma_t for m in media], [m.sigma_s for m in media], kernel=kernel)
    return b, media


def packed(b, media, rng):
    return np.concatenate([m.f + 0.1 * rng.standard_normal(m.N) for m in media])


@pytest.mark.parametrize("kernel", [P.VIE_KERNEL_AUTO, P.VIE_KERNEL_SYMMETRIC])
def test_small_uneven_batch_all_rows_and_single_grid_equality(kernel):
    ns = [1, 5, 17, 40, 23]
    b, media = make_batch(ns, kernel=kernel)
    g = packed(b, media, np.random.default_rng(0))
    y = torch.empty(b.total, dtype=torch.float64, device="cuda:0")
    P.vie_batch_apply(b, P.VIE_OP_K_SIGMA_S, dev(g), y)
    y = host(y)
    for i, m in enumerate(media):
        sl = slice(b.offsets[i], b.offsets[i + 1])
        want = O.apply(2, m.sigma_t, m.sigma_s, g[sl])
        assert rel_l2(y[sl], want) < TOL, ns[i]
        # each grid runs the kernel a single-grid handle with the same choice
        # takes (the displacement kernel for n = 5 .. 40 under AUTO, the
        # tile-pair kernel otherwise): the same arithmetic
        h = P.vie_create(2, m.n, m.sigma_t, m.sigma_s, kernel=kernel)
        y1 = torch.empty(m.N, dtype=torch.float64, device="cuda:0")
        P.vie_apply(h, P.VIE_OP_K_SIGMA_S, dev(g[sl]), y1)
        if P.vie_get_kernel(h) == P.VIE_KERNEL_DISPLACEMENT:
            np.testing.assert_array_equal(y[sl], host(y1))      # exact fixed-point sums
        else:
            np.testing.assert_allclose(y[sl], host(y1), rtol=1e-12, atol=0)


def test_ops_graph_recapture_and_host_pointers():
    ns = [12, 30]
    b, media = make_batch(ns, seed0=400)
    rng = np.random.default_rng(1)
    gA, gB = packed(b, media, rng), packed(b, media, rng)
    yA = torch.empty(b.total, dtype=torch.float64, device="cuda:0")
    yB = torch.empty_like(yA)
    dA, dB = dev(gA), dev(gB)
    for op in (P.VIE_OP_I_MINUS_K, P.VIE_OP_A_RAW):
        P.vie_batch_apply(b, op, dA, yA)
        P.vie_batch_apply(b, op, dB, yB)      # new pointers: re-captured graph
        P.vie_batch_apply(b, op, dA, yA)      # and back
        yh = np.empty(b.total)
        P.vie_batch_apply(b, op, np.ascontiguousarray(gB), yh)
        for i, m in enumerate(media):
            sl = slice(b.offsets[i], b.offsets[i + 1])
            oop = O.OP_I_MINUS_K if op == P.VIE_OP_I_MINUS_K else O.OP_A_RAW
            assert rel_l2(host(yA)[sl], O.apply(2, m.sigma_t, m.sigma_s, gA[sl], op=oop)) < TOL
            assert rel_l2(yh[sl], O.apply(2, m.sigma_t, m.sigma_s, gB[sl], op=oop)) < TOL
        np.testing.assert_array_equal(yh, host(yB))


@pytest.mark.parametrize("kernel", [P.VIE_KERNEL_AUTO, P.VIE_KERNEL_SYMMETRIC])
def test_several_sources_per_medium(kernel):
    # the R-source form: [nrhs][total] packed sources in one graph replay;
    # each source's result equals its single-source apply (the same launches)
    ns = [9, 24, 40]
    b, media = make_batch(ns, seed0=450, kernel=kernel)
    rng = np.random.default_rng(4)
    R = 5
    G = np.stack([packed(b, media, rng) for _ in range(R)])
    Y = torch.empty(R * b.total, dtype=torch.float64, device="cuda:0")
    P.vie_batch_apply(b, P.VIE_OP_K_SIGMA_S, dev(G.ravel()), Y, nrhs=R)
    Y = host(Y).reshape(R, b.total)
    one = torch.empty(b.total, dtype=torch.float64, device="cuda:0")
    for r in range(R):
        P.vie_batch_apply(b, P.VIE_OP_K_SIGMA_S, dev(G[r]), one)
        np.testing.assert_array_equal(Y[r], host(one))
        for i, m in enumerate(media):
            sl = slice(b.offsets[i], b.offsets[i + 1])
            assert rel_l2(Y[r][sl], O.apply(2, m.sigma_t, m.sigma_s, G[r][sl])) < TOL
    Yh = np.empty((R, b.total))                 # host buffers: the staging grows
    P.vie_batch_apply(b, P.VIE_OP_K_SIGMA_S, np.ascontiguousarray(G), Yh, nrhs=R)
    np.testing.assert_array_equal(Yh, Y)
    for bad in (0, 4097):
        with pytest.raises(P.VieError) as e:
            P.vie_batch_apply(b, P.VIE_OP_K_SIGMA_S, dev(G.ravel()), torch.empty(R * b.total, dtype=torch.float64,
                                                                                   device="cuda:0"), nrhs=bad)
        assert e.value.status == P.vie.VIE_ERR_INVALID_ARG


def test_autotune_and_cache(tmp_path):
    ns = [33, 64, 20]
    b, media = make_batch(ns, seed0=500)
    cache = str(tmp_path / "tune.txt")
    cfg = P.vie_batch_autotune(b, cache)
    assert cfg[0] in (2, 4, 8) and cfg[1] in (0, 1)
    assert os.path.exists(cache) and open(cache).read().strip()
    b2, _ = make_batch(ns, seed0=500)
    assert P.vie_batch_autotune(b2, cache) == cfg      # read back, no timing
    g = packed(b, media, np.random.default_rng(2))
    y = np.empty(b.total)
    P.vie_batch_apply(b, P.VIE_OP_K_SIGMA_S, np.ascontiguousarray(g), y)
    for i, m in enumerate(media):
        sl = slice(b.offsets[i], b.offsets[i + 1])
        assert rel_l2(y[sl], O.apply(2, m.sigma_t, m.sigma_s, g[sl])) < TOL


@pytest.mark.parametrize("kernel", [P.VIE_KERNEL_AUTO, P.VIE_KERNEL_SYMMETRIC])
def test_sixteen_uneven_grids_64_to_256_sampled_rows(kernel):
    ns = V.uneven_grid_sizes()
    media = V.uneven_media()
    b = P.vie_batch_create(ns, [m.sigma_t for m in media], [m.sigma_s for m in media], kernel=kernel)
    g = np.concatenate([m.f for m in media])
    y = torch.empty(b.total, dtype=torch.float64, device="cuda:0")
    P.vie_batch_apply(b, P.VIE_OP_K_SIGMA_S, dev(g), y)
    y = host(y)
    rng = np.random.default_rng(3)
    # 64, 154, 218 (the displacement kernel under AUTO; the largest lattice in
    # shared memory for the tile pairs), 230 and 256 (under AUTO the displacement
    # kernel with its lattice in global memory; tile pairs with sigma from global)
    for i in (0, 7, 12, 13, 15):
        m = media[i]
        sl = slice(b.offsets[i], b.offsets[i + 1])
        rows = np.unique(np.concatenate([rng.choice(m.N, 6, replace=False), [0, m.N - 1]]))
        want = O.apply(2, m.sigma_t, m.sigma_s, g[sl], rows=rows)
        assert rel_l2(y[sl][rows], want) < TOL, ns[i]
