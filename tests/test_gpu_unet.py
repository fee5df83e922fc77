"""The learned preconditioner's network on the GPU vs the FP64 reference, and FGMRES."""
import numpy as np
import pytest

import oracle as O
import vie_synth as V
from oracle import unet as R

torch = pytest.importorskip("torch")
import paper_1610_00835_gb300 as P  # noqa: E402
from gpu_util import dev, host, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu


def ref_params(u, levels, channels):
    flat = P.vie_unet_get_params(u).astype(np.float64)
    out, off = [], 0
    for co, ci, k in R.layer_shapes(levels, channels):
        nw = co * ci * k * k
        out.append(flat[off:off + nw].reshape(co, ci, k, k))
        off += nw
        out.append(flat[off:off + co])
        off += co
    assert off == flat.size
    return out


@pytest.mark.parametrize("levels,channels,n,B", [(1, 4, 8, 1), (3, 8, 16, 2), (4, 32, 32, 2),
                                                 (2, 5, 24, 3)])
def test_forward_and_gradients_match_reference(levels, channels, n, B):
    u = P.vie_unet_create(levels, channels, seed=11)
    rng = np.random.default_rng(levels)
    params = P.vie_unet_get_params(u)
    params = params + 0.02 * rng.standard_normal(params.size).astype(np.float32)  # nonzero biases
    P.vie_unet_set_params(u, params)
    x = rng.standard_normal((B, 3, n, n)).astype(np.float32)
    t = rng.standard_normal((B, 1, n, n)).astype(np.float32)
    o = torch.empty(B * n * n, dtype=torch.float32, device="cuda:0")
    P.vie_unet_forward(u, dev(x.ravel(), torch.float32), o, B, n)
    pr = ref_params(u, levels, channels)
    loss_ref, grads_ref, o_ref = R.loss_and_grads(pr, x.astype(np.float64), t.astype(np.float64), levels)
    assert rel_l2(host(o), o_ref.ravel()) < 1e-5
    loss, g = P.vie_unet_loss_grad(u, dev(x.ravel(), torch.float32), dev(t.ravel(), torch.float32), B, n)
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    off = 0
    for gr in grads_ref:
        k = gr.size
        assert rel_l2(g[off:off + k], gr.ravel()) < 1e-4
        off += k
    # BF16 weights for inference: close to the FP32 forward
    ob = torch.empty_like(o)
    P.vie_unet_forward(u, dev(x.ravel(), torch.float32), ob, B, n, use_bf16=True)
    assert rel_l2(host(ob), host(o)) < 2e-2


@pytest.mark.parametrize("B", [1, 2, 3])
def test_forward_at_256_on_every_tile_shape(B):
    # the convolution's tile (rows x 32 columns x output channels per CTA)
    # follows the grid: at 256^2 B = 3 takes 16 x 32 x 32, B = 2 16 x 32 x 16,
    # B = 1 8 x 32 x 16, and the coarse levels go down to 8 x 32 x 8.  Each
    # output sums its channels and taps in one order whatever the tile, so a
    # batch equals its images run one by one, bit for bit.
    levels, channels, n = 4, 32, 256
    u = P.vie_unet_create(levels, channels, seed=21)
    rng = np.random.default_rng(30 + B)
    params = P.vie_unet_get_params(u)
    P.vie_unet_set_params(u, params + 0.02 * rng.standard_normal(params.size).astype(np.float32))
    x = rng.standard_normal((B, 3, n, n)).astype(np.float32)
    o = torch.empty(B * n * n, dtype=torch.float32, device="cuda:0")
    P.vie_unet_forward(u, dev(x.ravel(), torch.float32), o, B, n)
    o_ref, _ = R.forward(ref_params(u, levels, channels), x.astype(np.float64), levels)
    assert rel_l2(host(o), o_ref.ravel()) < 1e-5
    one = torch.empty(n * n, dtype=torch.float32, device="cuda:0")
    for i in range(B):
        P.vie_unet_forward(u, dev(x[i].ravel(), torch.float32), one, 1, n)
        np.testing.assert_array_equal(host(one), host(o)[i * n * n:(i + 1) * n * n])


def _bf16_case(levels, n, B, seed):
    u = P.vie_unet_create(levels, 32, seed=seed)
    rng = np.random.default_rng(seed + n)
    params = P.vie_unet_get_params(u)
    P.vie_unet_set_params(u, params + 0.02 * rng.standard_normal(params.size).astype(np.float32))
    x = rng.standard_normal((B, 3, n, n)).astype(np.float32)
    o = torch.empty(B * n * n, dtype=torch.float32, device="cuda:0")
    P.vie_unet_forward(u, dev(x.ravel(), torch.float32), o, B, n, use_bf16=True)
    pr = ref_params(u, levels, 32)
    want, _ = R.forward(pr, x.astype(np.float64), levels, bf16=True)
    exact, _ = R.forward(pr, x.astype(np.float64), levels)
    return host(o), want.ravel(), exact.ravel()


@pytest.mark.parametrize("n,B", [(8, 1), (12, 2), (40, 1), (64, 2)])
def test_bf16_convolutions_on_tensor_cores_match_the_rounded_reference(n, B):
    # one level, 32 channels: a 3 -> 32 convolution (K = 27, one 64-wide K
    # block) and a 32 -> 32 one (K = 288: five blocks through the two-stage
    # ring) on the tensor cores, in 128-pixel tiles (64, 144, 1600, 4096
    # pixels: ragged and whole).  The first convolution's input is the same
    # FP32 array on both sides: its products agree to FP32 accumulation.  The
    # second's input is the first's output, FP32 here and FP64 there; where
    # one of its ~10^4..10^5 values lies within ~1e-7 of a BF16 tie the two
    # round it apart (a 2^-8 jump, about one case per 50k values), which moves
    # the outputs around that pixel by ~1e-4.  Everywhere else the results
    # agree to 1e-5.  A wrong rounding mode (~2e-3) or a lost K block (~1e-1)
    # fails both checks.
    got, want, _ = _bf16_case(1, n, B, seed=41)
    assert rel_l2(got, want) < 2e-4
    close = np.abs(got - want) <= 1e-5 * np.abs(want).max()
    assert close.mean() >= 0.98


@pytest.mark.parametrize("n,B", [(32, 2), (256, 1)])
def test_bf16_forward_on_tensor_cores_deep_network(n, B):
    # four levels (64 -> 32 decoder convolutions, K = 576, and coarse grids of
    # 16 pixels).  Deeper in the network the FP32 activations of the GPU and
    # the FP64 ones of the reference differ by ~1e-7, and a value that close
    # to a BF16 tie rounds differently on the two sides: a jump of 2^-8 that
    # the next layers spread over a patch.  So the deep forward is held to
    # the BF16 arithmetic's own scale: against the rounded reference, and
    # against the exact forward within the BF16 forward's own error (the
    # bound the CUDA-core BF16-weight forward is held to as well).
    got, want, exact = _bf16_case(4, n, B, seed=43)
    assert rel_l2(got, want) < 1e-2
    assert rel_l2(got, exact) < 2e-2


def test_training_reduces_loss():
    u = P.vie_unet_create(3, 8, seed=3)
    rng = np.random.default_rng(5)
    n, B = 16, 4
    x = dev(rng.standard_normal((B, 3, n, n)).ravel(), torch.float32)
    t = dev(np.tile(np.sin(np.linspace(0, 3, n))[None, None, :, None], (B, 1, 1, n)).ravel(), torch.float32)
    losses = [P.vie_unet_train_step(u, x, t, B, n, 3e-3) for _ in range(150)]
    assert losses[-1] < 0.2 * losses[0]


def test_save_load_roundtrip(tmp_path):
    u = P.vie_unet_create(2, 4, seed=1)
    path = str(tmp_path / "net.bin")
    P.vie_unet_save(u, path)
    v = P.vie_unet_create(2, 4, seed=2)
    P.vie_unet_load(v, path)
    np.testing.assert_array_equal(P.vie_unet_get_params(u), P.vie_unet_get_params(v))
    w = P.vie_unet_create(3, 4, seed=2)
    with pytest.raises(P.VieError):
        P.vie_unet_load(w, path)


@pytest.mark.parametrize("scale", [0.0, 1.0, 50.0])
def test_fgmres_converges_with_any_network(scale):
    # an untrained (scale 1), zero (scale 0: M = I) or wild (scale 50) network:
    # flexible GMRES or its plain fallback still reaches the tolerance
    n = 32
    m = V.heterogeneous_2d(n=n)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    u = P.vie_unet_create(4, 8, seed=7)
    P.vie_unet_set_params(u, P.vie_unet_get_params(u) * scale)
    P.vie_set_preconditioner(h, u)
    U = np.zeros(m.N)
    rep = P.vie_solve_gmres(h, m.f, U, rtol=1e-8)
    assert rep["converged"] and rep["precond_iters"] >= 1
    phi = O.apply(2, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW)
    assert rel_l2(U, O.lu_solve(2, m.sigma_t, m.sigma_s, phi)) < 1e-5
    P.vie_set_preconditioner(h, None)
    U2 = np.zeros(m.N)
    rep2 = P.vie_solve_gmres(h, m.f, U2, rtol=1e-8)
    assert rep2["precond_iters"] == 0


def test_checkpoint_resumes_adam_where_it_stopped(tmp_path):
    # three Adam steps, save, three more; a second network loaded from the
    # checkpoint takes the same three steps: both end with the same
    # parameters.  A restart from zero moments would take the fourth step with
    # a different effective rate (|update| ~ lr for every parameter).
    n, B = 16, 2
    rng = np.random.default_rng(17)
    x = dev(rng.standard_normal((B, 3, n, n)).ravel(), torch.float32)
    t = dev(rng.standard_normal((B, n, n)).ravel(), torch.float32)
    a = P.vie_unet_create(3, 8, seed=5)
    for _ in range(3):
        P.vie_unet_train_step(a, x, t, B, n, 1e-3)
    path = str(tmp_path / "ckpt.bin")
    P.vie_unet_save(a, path)
    assert P.vie_unet_train_state(a) == 3
    b = P.vie_unet_create(3, 8, seed=99)
    P.vie_unet_load(b, path)
    assert P.vie_unet_train_state(b) == 3
    np.testing.assert_array_equal(P.vie_unet_get_params(a), P.vie_unet_get_params(b))
    for _ in range(3):
        P.vie_unet_train_step(a, x, t, B, n, 1e-3)
        P.vie_unet_train_step(b, x, t, B, n, 1e-3)
    pa, pb = P.vie_unet_get_params(a), P.vie_unet_get_params(b)
    moved = np.abs(pa - P.vie_unet_get_params(P.vie_unet_create(3, 8, seed=5))).max()
    assert np.abs(pa - pb).max() <= 1e-4 * moved
    # a parameter-only start (moments and step reset) ends elsewhere
    c = P.vie_unet_create(3, 8, seed=99)
    P.vie_unet_set_params(c, P.vie_unet_get_params(b) * 0 + np.fromfile(path, dtype=np.float32)[6:6 + pa.size])
    for _ in range(3):
        P.vie_unet_train_step(c, x, t, B, n, 1e-3)
    assert np.abs(P.vie_unet_get_params(c) - pa).max() > 10 * np.abs(pa - pb).max()


@pytest.mark.parametrize("n,B", [(32, 2), (256, 1)])
def test_bf16_forward_every_layer_matches_the_rounded_reference(n, B):
    # the 4-level BF16 forward layer by layer: each convolution's output from
    # the tensor cores against the FP64 convolution of the same FP32 input with
    # the BF16 inference rounding (input and weights rounded to BF16, relu after
    # every 3x3 layer, the 1x1 head on FP32 activations).  Both sides round the
    # same input, so only the FP32 accumulation differs: every layer, the
    # encoder's 3 -> 32 and 32 -> 32, the decoder's 64 -> 32 (K = 576) at every
    # resolution down to the coarsest and the head, is held to 1e-5.
    levels, C = 4, 32
    u = P.vie_unet_create(levels, C, seed=51)
    rng = np.random.default_rng(n + B)
    params = P.vie_unet_get_params(u)
    P.vie_unet_set_params(u, params + 0.02 * rng.standard_normal(params.size).astype(np.float32))
    x = rng.standard_normal((B, 3, n, n)).astype(np.float32)
    o = torch.empty(B * n * n, dtype=torch.float32, device="cuda:0")
    P.vie_unet_forward(u, dev(x.ravel(), torch.float32), o, B, n, use_bf16=True)
    pr = ref_params(u, levels, C)
    shapes = R.layer_shapes(levels, C)
    res = [n >> l for l in range(levels) for _ in range(2)] + \
          [n >> l for l in range(levels - 2, -1, -1) for _ in range(2)] + [n]
    assert len(res) == len(shapes)
    for i, ((co, ci, k), H) in enumerate(zip(shapes, res)):
        inp = np.empty((B, ci, H, H), dtype=np.float32)
        out = np.empty((B, co, H, H), dtype=np.float32)
        P.vie_unet_layer_io(u, i, None if i == 0 else inp, out)
        if i == 0:
            inp = x
        w, b = pr[2 * i], pr[2 * i + 1]
        xi = inp.astype(np.float64)
        want = R.conv(R.round_bf16(xi) if k == 3 else xi, R.round_bf16(w), b)
        if k == 3:
            want = np.maximum(want, 0)
        assert rel_l2(out.ravel(), want.ravel()) < 1e-5, (i, co, ci, H)


@pytest.mark.parametrize("nrhs", [1, 3])
def test_network_on_diffusion_converges_with_any_network(nrhs):
    # the network as a correction of the diffusion preconditioner: with an
    # untrained network (or a zero one, M = D) FGMRES still reaches the
    # tolerance, one source or several in lockstep, and matches the LU solution
    # (optically thin cells, where the diffusion approximation holds)
    n = 32
    m = V.heterogeneous_2d(n=n, seed=8600)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    F = V.bump_sources(2, n, nrhs, seed=81)
    phi = [O.apply(2, m.sigma_t, m.sigma_s, f, op=O.OP_A_RAW) for f in F]
    K = O.k_matrix(2, m.sigma_t, m.sigma_s)
    want = [np.linalg.solve(np.eye(m.N) - K, p) for p in phi]
    for scale in (0.0, 1.0):
        u = P.vie_unet_create(4, 8, seed=7)
        P.vie_unet_set_params(u, P.vie_unet_get_params(u) * scale)
        P.vie_set_preconditioner_on_diffusion(h, u)
        U = np.zeros(nrhs * m.N)
        reps = P.vie_solve_gmres(h, F.ravel(), U, rtol=1e-8, nrhs=nrhs)
        reps = reps if nrhs > 1 else [reps]
        for r in range(nrhs):
            assert reps[r]["converged"] and reps[r]["precond_iters"] >= 1
            assert rel_l2(U[r * m.N:(r + 1) * m.N], want[r]) < 1e-5
    P.vie_set_preconditioner_on_diffusion(h, None)
    U = np.zeros(m.N)
    assert P.vie_solve_gmres(h, F[0], U, rtol=1e-8)["precond_iters"] == 0
