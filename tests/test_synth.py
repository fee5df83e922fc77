"""The seeded input generators that the oracle and the CUDA path share."""
import numpy as np

import vie_synth as V


def test_splitmix64_published_outputs():
    # the first outputs of SplitMix64 from state 0
    r = V.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = V.SplitMix64(12345)
    x = np.array([u.uniform() for _ in range(10000)])
    assert x.min() >= 0.0 and x.max() < 1.0 and abs(x.mean() - 0.5) < 0.02


def test_uneven_grid_sizes_and_media():
    ns = V.uneven_grid_sizes()
    assert ns == [64, 77, 90, 102, 115, 128, 141, 154, 166, 179, 192, 205, 218, 230, 243, 256]
    assert sum(n ** 4 for n in ns) == 19376528582
    a, b = V.uneven_media(), V.uneven_media()
    assert [m.n for m in a] == ns
    assert all(np.array_equal(p.sigma_t, q.sigma_t) and np.array_equal(p.f, q.f) for p, q in zip(a, b))


def test_cell_centres_and_index_convention():
    x = V.cell_centres(2, 4)
    assert x.shape == (16, 2)
    np.testing.assert_allclose(x[1], [0.375, 0.125])     # j = ix + n iy: x fastest
    np.testing.assert_allclose(x[4], [0.125, 0.375])
    x3 = V.cell_centres(3, 2)
    np.testing.assert_allclose(x3[4], [0.25, 0.25, 0.75])


def test_direction_sets_are_unit_vectors():
    d = V.fibonacci_directions(128)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(d[:, 2], 1 - (2 * np.arange(128) + 1) / 128, rtol=0, atol=1e-15)
    c = V.circle_directions(12)
    np.testing.assert_allclose(np.linalg.norm(c, axis=1), 1.0, rtol=0, atol=1e-15)
    assert abs(c.sum(axis=0)).max() < 1e-12


def test_media_are_seeded_and_positive():
    m1 = V.heterogeneous_2d(n=32)
    m2 = V.heterogeneous_2d(n=32)
    assert np.array_equal(m1.sigma_t, m2.sigma_t)
    assert (m1.sigma_t >= 1.0).all()
    np.testing.assert_allclose(m1.sigma_s, 0.9 * m1.sigma_t, rtol=1e-15)
    m3 = V.heterogeneous_3d(n=8)
    np.testing.assert_allclose(m3.sigma_s, 0.8 * m3.sigma_t, rtol=1e-15)
    assert not np.array_equal(V.heterogeneous_2d(n=32, seed=V.seed_for(2, 1)).sigma_t, m1.sigma_t)
