"""The library's caching device allocator (include/vie.h, vie_release_memory):
handles created per solve reuse the buffers of destroyed ones, give the same
results, and vie_release_memory returns the cached buffers to CUDA."""
import numpy as np
import pytest

import vie_synth as V

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1610_00835_gb300")

pytestmark = pytest.mark.gpu


def solve_once(m):
    h = P.vie_create(2, m.n, m.sigma_t, m.sigma_s)
    U = np.zeros(m.N)
    rep = P.vie_solve_gmres(h, m.f, U, rtol=1e-8)
    P.vie_destroy(h)
    return U, rep


def test_handles_reuse_cached_buffers_and_release_returns_them():
    m = V.heterogeneous_2d(n=64, seed=4401)
    U0, rep0 = solve_once(m)
    assert rep0["converged"]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(4):
        U, rep = solve_once(m)
        assert rep["iters"] == rep0["iters"]
        assert np.array_equal(U, U0)  # the same kernels on reused buffers: the same bits
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    # later handles took the cached buffers of the first: no new device memory
    assert free1 >= free0 - (8 << 20)
    P.vie_release_memory()
    free2 = torch.cuda.mem_get_info()[0]
    # the destroyed handles' buffers (the Krylov basis alone is 2 MB) went back to CUDA
    assert free2 >= free1 + (1 << 20)
    # and the next handle allocates afresh and still gives the same bits
    U, _ = solve_once(m)
    assert np.array_equal(U, U0)
