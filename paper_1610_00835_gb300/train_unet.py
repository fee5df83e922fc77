"""Train the learned right preconditioner on solves generated by the method.

Data: `--samples` random 2D media on an n x n grid, seeds 5000 + i (a third
physical solves b = phi, two thirds manufactured pairs b = (I - K) w), from the
`--family` "diffusive" (vie_synth.diffusive_training_medium: sigma_s = s (1 +
bumps), s log-uniform in [5, 30], mu_a in [0.1, 0.5], the strongly scattering
regime of the paper's preconditioning experiments) or "thin"
(vie_synth.random_training_medium: sigma_s / sigma_t in [0.5, 0.95]).  Even samples use
the physical right-hand side phi = A f, odd ones a random smooth field b
(vie_synth.random_rhs, seed 7000 + i).  Each (I - K) U = b is solved with the
assembled BF16 hi/lo operator and FP64 GMRES to 1e-8.  Network input
(sigma_t / s_ref, sigma_s / s_ref, b / rms(b)), target (U - b) / rms(b): the
network learns the smooth part of (I - K)^{-1} b (the preconditioner is
M(b) = b + rms(b) Net(...)).

Training: Adam, batch 16, cosine learning-rate decay, the library's own
forward and backward kernels.  Then, on held-out media at `--eval-n` (seeds
9000 + i), one solve with plain GMRES and one with FGMRES + the network, both
to 1e-6 with the assembled operator; prints iterations and times.

    python -m paper_1610_00835_gb300.train_unet --out paper_1610_00835_gb300/data/unet_l4_c32.bin
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import vie_synth as V  # noqa: E402

S_REF = 5.0
FAMILIES = {"thin": V.random_training_medium, "diffusive": V.diffusive_training_medium}


def make_sample(P, torch, i, n, dev, family="diffusive", base="identity"):
    """Sample i: kind i % 3 = 0 a physical solve (b = phi = A f, U by GMRES to
    1e-6); 1 and 2 a manufactured pair (U = w a random smooth / rough field,
    b = (I - K) w by one apply), which covers the residual-like vectors a
    Krylov method feeds to its preconditioner.  The target is (U - z0) / rms(b)
    with z0 = b (base "identity": M(b) = b + rms(b) Net) or z0 the diffusion
    preconditioner's D(b) (base "diffusion": M(b) = D(b) + rms(b) Net)."""
    m = FAMILIES[family](n, 5000 + i)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    kind = i % 3
    rep = {"iters": 0, "converged": 1}
    if kind == 0:
        P.vie_assemble(h, P.VIE_OPERATOR_BF16X3)
        f = torch.as_tensor(m.f, dtype=torch.float64, device=dev)
        b = torch.empty_like(f)
        P.vie_apply(h, P.VIE_OP_A_RAW, f, b)
        U = torch.empty_like(b)
        rep = P.vie_solve_gmres(h, b, U, rtol=1e-6, restart=128, maxit=1500, rhs_is_phi=True,
                                raise_on_nonconvergence=False)
    else:
        width = (0.05, 0.3) if kind == 1 else (0.01, 0.05)
        U = torch.as_tensor(V.random_field(n, 7000 + i, width=width), dtype=torch.float64,
                            device=dev)
        b = torch.empty_like(U)
        P.vie_apply(h, P.VIE_OP_I_MINUS_K, U, b)
    z0 = b
    if base == "diffusion" and rep["converged"]:
        P.vie_set_diffusion_preconditioner(h)
        z0 = torch.empty_like(b)
        P.vie_diffusion_precondition(h, b, z0)
    P.vie_destroy(h)
    if not rep["converged"]:
        return None, None, rep["iters"]
    rms = torch.sqrt(torch.mean(b * b))
    x = torch.stack([torch.as_tensor(m.sigma_t, device=dev) / S_REF,
                     torch.as_tensor(m.sigma_s, device=dev) / S_REF, b / rms]).float()
    t = ((U - z0) / rms).float()
    return x.reshape(-1), t, rep["iters"]


def evaluate(P, torch, net, n, count, dev, rtol=1e-6, family="diffusive", base="identity"):
    rows = []
    for i in range(count):
        m = FAMILIES[family](n, 9000 + i)
        h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
        P.vie_assemble(h, P.VIE_OPERATOR_BF16X3)
        f = torch.as_tensor(m.f, dtype=torch.float64, device=dev)
        res = {}
        cases = (("plain", None), ("learned", net)) if base == "identity" else \
            (("plain", None), ("diffusion", "diffusion"), ("learned", net))
        for name, pre in cases:
            P.vie_set_preconditioner(h, None)
            if pre == "diffusion":
                P.vie_set_diffusion_preconditioner(h)
            elif pre is not None and base == "diffusion":
                P.vie_set_preconditioner_on_diffusion(h, pre, S_REF)
            elif pre is not None:
                P.vie_set_preconditioner(h, pre, S_REF)
            U = torch.empty_like(f)
            P.vie_solve_gmres(h, f, U, rtol=rtol, restart=128, maxit=3000,
                              raise_on_nonconvergence=False)          # warm-up (allocations)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = P.vie_solve_gmres(h, f, U, rtol=rtol, restart=128, maxit=3000,
                                    raise_on_nonconvergence=False)
            torch.cuda.synchronize()
            res[name] = {"iters": rep["iters"], "ms": 1e3 * (time.perf_counter() - t0),
                         "relres": rep["relres"], "fell_back": rep["fell_back"],
                         "converged": rep["converged"]}
        P.vie_set_preconditioner(h, None)
        P.vie_set_diffusion_preconditioner(h, False)
        P.vie_destroy(h)
        rows.append(res)
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=2000)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--levels", type=int, default=4)
    ap.add_argument("--channels", type=int, default=32)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--eval-n", type=int, default=256)
    ap.add_argument("--eval-count", type=int, default=8)
    ap.add_argument("--family", choices=sorted(FAMILIES), default="diffusive")
    ap.add_argument("--base", choices=["identity", "diffusion"], default="identity",
                    help="what the network corrects: the identity (M(b) = b + rms(b) Net) or the "
                         "diffusion preconditioner (M(b) = D(b) + rms(b) Net)")
    ap.add_argument("--out", default=None)
    ap.add_argument("--report", default=None)
    ap.add_argument("--checkpoint", default=None,
                    help="after every epoch, save the network with its optimizer state here (and the "
                         "epoch and the shuffling generator's state beside it, PATH.json)")
    ap.add_argument("--resume", action="store_true",
                    help="continue from --checkpoint: the data are drawn again from their seeds, the "
                         "network, Adam state, epoch and shuffling resume where the checkpoint stopped")
    args = ap.parse_args(argv)
    import torch
    import paper_1610_00835_gb300 as P

    dev = "cuda:0"
    t0 = time.perf_counter()
    X = torch.empty(args.samples, 3 * args.n * args.n, dtype=torch.float32, device=dev)
    Wt = torch.empty(args.samples, dtype=torch.float32, device=dev)
    T = torch.empty(args.samples, args.n * args.n, dtype=torch.float32, device=dev)
    iters, kept, i = [], 0, 0
    while kept < args.samples and i < 2 * args.samples:
        x, t, it = make_sample(P, torch, i, args.n, dev, args.family, args.base)
        i += 1
        iters.append(it)
        if x is None:
            continue
        X[kept], T[kept] = x, t
        Wt[kept] = 1.0 / (torch.mean(t.double() ** 2) + 1e-12)   # relative error per sample
        kept += 1
    X, T, Wt = X[:kept], T[:kept], Wt[:kept]
    args.samples = kept
    gen_s = time.perf_counter() - t0
    print(json.dumps({"phase": "data", "samples": kept, "tried": i, "seconds": gen_s,
                      "gmres_iters_mean": float(np.mean(iters)),
                      "gmres_iters_max": int(np.max(iters))}), flush=True)

    hold = max(1, args.samples // 32)
    ntrain = args.samples - hold
    net = P.vie_unet_create(args.levels, args.channels, seed=args.seed)
    rng = np.random.default_rng(args.seed)
    steps_per_epoch = ntrain // args.batch
    total = steps_per_epoch * args.epochs
    step = 0
    first_epoch = 0
    if args.resume:
        if not args.checkpoint:
            raise SystemExit("--resume needs --checkpoint")
        P.vie_unet_load(net, args.checkpoint)
        with open(args.checkpoint + ".json") as fh:
            side = json.load(fh)
        first_epoch = side["epoch"] + 1
        step = side["step"]
        rng.bit_generator.state = side["rng"]
        if P.vie_unet_train_state(net) != step:
            raise SystemExit("checkpoint and its side file disagree on the step count")
    t1 = time.perf_counter()
    for ep in range(first_epoch, args.epochs):
        perm = torch.as_tensor(rng.permutation(ntrain), device=dev)
        losses = []
        for s in range(steps_per_epoch):
            idx = perm[s * args.batch:(s + 1) * args.batch]
            xb = X[idx].contiguous().reshape(-1)
            tb = T[idx].contiguous().reshape(-1)
            lr = 1e-5 + 0.5 * (args.lr - 1e-5) * (1 + math.cos(math.pi * step / total))
            wb = Wt[idx].contiguous()
            losses.append(P.vie_unet_train_step(net, xb, tb, args.batch, args.n, lr, weights=wb))
            step += 1
        vx = X[ntrain:].contiguous().reshape(-1)
        vt = T[ntrain:].contiguous().reshape(-1)
        vloss, _ = P.vie_unet_loss_grad(net, vx, vt, hold, args.n)
        tvar = float(torch.mean(T[ntrain:] ** 2))  # unweighted validation error
        print(json.dumps({"phase": "train", "epoch": ep, "loss": float(np.mean(losses)),
                          "val_loss": vloss, "val_rel": math.sqrt(vloss / tvar)}), flush=True)
        if args.checkpoint:
            os.makedirs(os.path.dirname(os.path.abspath(args.checkpoint)), exist_ok=True)
            P.vie_unet_save(net, args.checkpoint)
            with open(args.checkpoint + ".json", "w") as fh:
                json.dump({"epoch": ep, "step": step, "rng": rng.bit_generator.state}, fh)
    train_s = time.perf_counter() - t1
    if args.out:
        os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
        P.vie_unet_save(net, args.out)
    rows = (evaluate(P, torch, net, args.eval_n, args.eval_count, dev, family=args.family, base=args.base)
            if args.eval_count else [])
    summary = {"phase": "eval", "n": args.eval_n, "train_seconds": train_s, "data_seconds": gen_s,
               "plain_iters": [r["plain"]["iters"] for r in rows],
               "learned_iters": [r["learned"]["iters"] for r in rows],
               "plain_ms": [r["plain"]["ms"] for r in rows],
               "learned_ms": [r["learned"]["ms"] for r in rows],
               "diffusion_iters": [r["diffusion"]["iters"] for r in rows if "diffusion" in r],
               "diffusion_ms": [r["diffusion"]["ms"] for r in rows if "diffusion" in r],
               "fell_back": [r["learned"]["fell_back"] for r in rows],
               "converged": [[r["plain"]["converged"], r["learned"]["converged"]] for r in rows]}
    print(json.dumps(summary), flush=True)
    if args.report:
        with open(args.report, "w") as fh:
            json.dump(summary, fh)
    return 0


if __name__ == "__main__":
    sys.exit(main())
