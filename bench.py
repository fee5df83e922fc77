"""Benchmark of the VIE hot path on one GB300 (or N replicas under torchrun).

Workload (one "step"): the 2D heterogeneous 128x128 medium (16384 unknowns,
sigma_t = 1 + 4 seeded Gaussian bumps, sigma_s = 0.9 sigma_t, bilinear
sigma_t, tau by a 64-step march, FP32 kernel tiles), Gaussian source at the
centre: phi = A f, then FP64 GMRES(64) to 1e-6 relative residual, every
Arnoldi step one on-the-fly operator apply.  The medium's handle (sigma_t
staging, self-cell diagonal) is built once before timing; inputs sit in HBM.

value  = pairs evaluated per second over the whole job (n_apply * N^2 per
         step, summed over ranks) in Gpair/s.
e2e    = the same through the C ABI from host buffers: vie_create from host
         sigma_t/sigma_s, vie_solve_gmres with host f and host U (copies
         inside), vie_destroy; per step.
roofline: the pair kernel, bound by the FP32 pipe (it is issue-bound: the
         multiply-adds of the optical depths plus their loads and
         bookkeeping).  Algorithmic work = the multiply-adds of the tau sums
         by the method's own count (vie_get_kernel_work): for the
         displacement kernel sum_D |W_D| x pairs(D), W_D the per-cell sum of
         the S midpoint samples' bilinear weights.  Peak = SMs x 128 FP32
         FMA lanes x max SM clock.
cpu_baseline: the FP64 oracle's matrix-free apply on a bounded sample of
         target rows of the same medium, on the host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import vie_synth as V  # noqa: E402

METRIC = "VIE matvec Gpair/s; GMRES solve ms to 1e-6 rel. residual, plain vs chosen"
UNIT = "Gpair/s"
WORKLOAD = "2D heterogeneous 128x128, sigma_t = 1 + 4 seeded bumps, sigma_s = 0.9 sigma_t, S=64 march"
S_STEPS = 64
RTOL = 1e-6
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one cold-cache
# launch of each pair kernel on this workload, from one ncu capture of the
# kernel as it is now; an entry goes back to None whenever its kernel changes,
# until it is captured again.
PAIR_KERNEL_DRAM_BYTES = {1: 229376,     # k_pairs_sym<2,129,0>
                          2: 48577536}   # k_pairs_disp<141,12>: 48.47 MB read (the chunk records), 0.11 MB written
KERNEL_NAMES = {1: "k_pairs_sym<2,129,0>", 2: "k_pairs_disp<141,12>", 3: "k_pairs_f32"}


def nvtx_push(torch, name: str) -> None:
    """Mark a timed step for profilers (ncu --nvtx --nvtx-include timed_step/)."""
    try:
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop(torch) -> None:
    try:
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def medium(rank: int):
    return V.heterogeneous_2d(n=128, seed=V.seed_for(2, rank))


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def flush_l2(buf):
    buf.zero_()


def cpu_baseline_sample(m, seconds: float = 12.0) -> dict:
    """The oracle's apply on a bounded sample of target rows (host cores)."""
    import oracle as O
    g = m.f
    diag = O.selfcells(2, m.sigma_t)
    rows = np.arange(0, m.N, 997)[:8]
    t0 = time.perf_counter()
    O.apply(2, m.sigma_t, m.sigma_s, g, rows=rows, diag=diag)
    dt = time.perf_counter() - t0
    count = int(max(8, min(m.N, len(rows) * seconds / max(dt, 1e-3))))
    rows = np.linspace(0, m.N - 1, count).astype(np.int64)
    t0 = time.perf_counter()
    O.apply(2, m.sigma_t, m.sigma_s, g, rows=rows, diag=diag)
    dt = time.perf_counter() - t0
    out = {"value": len(rows) * m.N / dt / 1e9, "unit": UNIT, "cores": O.num_threads(),
           "kind": "oracle",
           "sample": f"{len(rows)} target rows x {m.N} sources of the 128x128 medium, "
                     f"S={S_STEPS}, FP64 matrix-free apply ({dt:.1f} s)"}
    # the same on one core (the paper's runs were single-threaded), a smaller sample
    threads = O.num_threads()
    O.set_threads(1)
    try:
        rows1 = np.linspace(0, m.N - 1, max(4, count // (4 * threads))).astype(np.int64)
        t0 = time.perf_counter()
        O.apply(2, m.sigma_t, m.sigma_s, g, rows=rows1, diag=diag)
        dt1 = time.perf_counter() - t0
    finally:
        O.set_threads(threads)
    out["one_core"] = {"value": len(rows1) * m.N / dt1 / 1e9, "unit": UNIT, "cores": 1,
                       "sample": f"{len(rows1)} target rows ({dt1:.1f} s)"}
    return out


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, timed on the host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O
    m = medium(0)
    diag = O.selfcells(2, m.sigma_t)
    per_step_rows = 24
    stride = m.N // per_step_rows
    times = []
    for it in range(args.warmup + args.steps):
        rows = (np.arange(per_step_rows) * stride + it) % m.N
        t0 = time.perf_counter()
        O.apply(2, m.sigma_t, m.sigma_s, m.f, rows=rows, diag=diag)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = per_step_rows * m.N * len(times) / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD + "; oracle apply on 24 target rows per step",
                   "l2": "not applicable (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"{per_step_rows} target rows x {m.N} sources per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def oracle_solution(rank: int):
    """The FP64 oracle's U for the benchmark medium (rank 0's seed), written by
    tests/golden/make_bench_solution.py; None for other media."""
    path = os.path.join(ROOT, "tests", "golden", "bench_U_2d_128.npy")
    if rank != 0 or not os.path.exists(path):
        return None
    return np.load(path)


def err_vs_oracle(U, U_or):
    if U_or is None:
        return None
    u = U.detach().cpu().numpy() if hasattr(U, "detach") else np.asarray(U)
    return float(np.linalg.norm(u - U_or) / np.linalg.norm(U_or))


def measure_assembled(P, torch, h, f_dev, U, flush, stream, args, operator, U_or, net=None, fft=False):
    """Assemble K once per step (one march per unordered pair; BF16 hi/lo or
    FP32), then FP64 GMRES(64) -- or FGMRES with the learned preconditioner --
    whose applies are HBM-bound products with the stored K (phi = K(f /
    sigma_s)).  Assembly is inside every timed step."""
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c = torch.cuda.Event(enable_timing=True)
    P.vie_set_preconditioner(h, net, 5.0)
    if fft:
        P.vie_set_fft_preconditioner(h)
    for _ in range(max(1, args.warmup)):
        P.vie_assemble(h, operator)
        P.vie_solve_gmres(h, f_dev, U, rtol=RTOL)
    ms, asm_ms, reps = [], [], []
    for _ in range(max(3, args.steps // 4)):
        flush_l2(flush)
        torch.cuda.synchronize()
        nvtx_push(torch, "assembled_step")
        a.record(stream)
        P.vie_assemble(h, operator)
        b.record(stream)
        rep = P.vie_solve_gmres(h, f_dev, U, rtol=RTOL, time_apply=True)
        c.record(stream)
        torch.cuda.synchronize()
        nvtx_pop(torch)
        ms.append(a.elapsed_time(c))
        asm_ms.append(a.elapsed_time(b))
        reps.append(rep)
    P.vie_set_preconditioner(h, None)
    P.vie_set_fft_preconditioner(h, False)
    P.vie_assemble(h, P.VIE_OPERATOR_OTF)
    last = reps[-1]
    name = {P.VIE_OPERATOR_BF16X3: "assembled BF16 hi/lo operator (row-major, 1.07 GB)",
            P.VIE_OPERATOR_FP32: "assembled FP32 operator (row-major, 1.07 GB)",
            P.VIE_OPERATOR_PAIRS32: "assembled FP32 pair weights (displacement-major, each unordered pair once, 0.54 GB)",
            P.VIE_OPERATOR_SYM32: "assembled FP32 A in symmetric grid-row blocks (each unordered pair of rows once, 0.54 GB)",
            P.VIE_OPERATOR_FMM: "FMM of Section 3.3, Chebyshev order 6, cached near-field and M2L blocks (0.09 GB)"}
    return {"solver": name[operator] + (" + FGMRES(64), learned U-Net preconditioner" if net is not None
                                        else " + FGMRES(64), FFT preconditioner" if fft
                                        else " + FP64 GMRES(64)"),
            "solve_ms": statistics.median(ms), "assemble_ms": statistics.median(asm_ms),
            "iters": last["iters"], "n_apply": last["n_apply"], "relres": last["relres"],
            "fell_back": last["fell_back"], "apply_ms": last["t_apply_ms"] / max(1, last["n_apply"]),
            "err_vs_oracle": err_vs_oracle(U, U_or)}


def measure_mii(P, torch, m, f_dev, flush, stream, args, local, rank, U_miii):
    """Approach M-ii (Section 3.2, Remark REM: NEW KERNEL) on the benchmark
    medium: the plain on-the-fly solve and the chosen assembled solve, each
    against the FP64 oracle's M-ii solution (tests/golden/bench_U_2d_128_mii.npy),
    and the relative difference from the M-iii solution (the discretisation
    change itself)."""
    hm = P.vie_create(2, m.n, m.sigma_t, m.sigma_s, steps=S_STEPS, device=local, disc=P.VIE_DISC_MII)
    U = torch.empty(m.N, dtype=torch.float64, device=f"cuda:{local}")
    path = os.path.join(ROOT, "tests", "golden", "bench_U_2d_128_mii.npy")
    U_or = np.load(path) if rank == 0 and os.path.exists(path) else None
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(max(1, args.warmup)):
        P.vie_solve_gmres(hm, f_dev, U, rtol=RTOL)
    ms, rep = [], None
    for _ in range(max(3, args.steps // 4)):
        flush_l2(flush)
        torch.cuda.synchronize()
        a.record(stream)
        rep = P.vie_solve_gmres(hm, f_dev, U, rtol=RTOL)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    plain = {"solver": "plain: FP64 GMRES(64), on-the-fly FP32 operator, M-ii weights",
             "solve_ms": statistics.median(ms), "iters": rep["iters"], "n_apply": rep["n_apply"],
             "relres": rep["relres"], "err_vs_oracle": err_vs_oracle(U, U_or)}
    chosen = measure_assembled(P, torch, hm, f_dev, U, flush, stream, args, P.VIE_OPERATOR_SYM32, U_or)
    P.vie_destroy(hm)
    return {"plain": plain, "chosen": chosen,
            "rel_diff_vs_m3_solution": err_vs_oracle(U_miii, err_ref(U)) if U_miii is not None else None,
            "oracle_U": "tests/golden/bench_U_2d_128_mii.npy (FP64 oracle, rtol 1e-11)"
            if U_or is not None else None}


def err_ref(U):
    return U.detach().cpu().numpy() if hasattr(U, "detach") else np.asarray(U)


def measure_bf16x3_product(P, torch, m, h, stream, args, local, nrhs=64):
    """Y = K G for 64 seeded bump sources with the assembled BF16 hi/lo K on
    the tensor cores (one launch for all 64 right-hand sides)."""
    N = m.N
    G = torch.as_tensor(V.bump_sources(2, m.n, nrhs, seed=V.seed_for(4)).ravel(),
                        dtype=torch.float64, device=f"cuda:{local}")
    Y = torch.empty_like(G)
    P.vie_assemble(h, P.VIE_OPERATOR_BF16X3)
    for _ in range(3):
        P.vie_apply(h, P.VIE_OP_K_SIGMA_S, G, Y, nrhs)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        P.vie_apply(h, P.VIE_OP_K_SIGMA_S, G, Y, nrhs)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    P.vie_assemble(h, P.VIE_OPERATOR_OTF)
    ldk = (N + 63) // 64 * 64
    # algorithmic bytes: K hi + lo once, G (FP64 in) and Y (FP64 out)
    traffic = 4.0 * N * ldk + 2 * 8.0 * nrhs * N
    peak = 6678.2
    try:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except (OSError, KeyError, ValueError):
        pass
    achieved = traffic / (ms * 1e-3) / 1e9
    return {"nrhs": nrhs, "ms": ms, "gpair_per_s": float(N) * N * nrhs / (ms * 1e-3) / 1e9,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "k_gemm_bf16x3 (+ split and finish kernels)",
                         "work": "4 B per K entry (hi + lo) + FP64 G and Y"}}


def measure_multi_source(P, torch, m, stream, local, nrhs=64):
    """The 64 seeded bump sources on the 128^2 medium solved to 1e-6: together
    (lockstep GMRES, one tensor-core product of all columns per Arnoldi step,
    assembled BF16 hi/lo K), with and without the learned preconditioner
    (one batched forward pass per step), against the same sources solved one
    at a time (the assembled operator's GEMV, and plain on-the-fly GMRES).
    Assembly (once per medium) is timed apart from the solves."""
    dev = f"cuda:{local}"
    N = m.N
    F = V.bump_sources(2, m.n, nrhs, seed=V.seed_for(4))
    f_all = torch.as_tensor(F.ravel(), dtype=torch.float64, device=dev)
    U_all = torch.empty_like(f_all)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=3):
        fn()
        ms, out = [], None
        for _ in range(reps):
            torch.cuda.synchronize()
            a.record(stream)
            out = fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms), out

    h = P.vie_create(2, m.n, m.sigma_t, m.sigma_s, steps=S_STEPS, device=local)
    asm_ms, _ = timed(lambda: P.vie_assemble(h, P.VIE_OPERATOR_BF16X3))
    lock_ms, reps = timed(lambda: P.vie_solve_gmres(h, f_all, U_all, rtol=RTOL, nrhs=nrhs))
    U_lock = U_all.detach().cpu().numpy().reshape(nrhs, N)
    net = P.vie_unet_create(4, 32, device=local)
    P.vie_unet_load(net, os.path.join(ROOT, "paper_1610_00835_gb300", "data", "unet_l4_c32.bin"))
    P.vie_set_preconditioner(h, net, 5.0)
    lockl_ms, repl = timed(lambda: P.vie_solve_gmres(h, f_all, U_all, rtol=RTOL, nrhs=nrhs))
    P.vie_set_preconditioner(h, None)
    P.vie_unet_destroy(net)
    u1 = torch.empty(N, dtype=torch.float64, device=dev)

    def one_by_one():
        its = []
        for r in range(nrhs):
            its.append(P.vie_solve_gmres(h, f_all[r * N:(r + 1) * N], u1, rtol=RTOL)["iters"])
        return its

    single_ms, single_its = timed(one_by_one, reps=1)
    P.vie_assemble(h, P.VIE_OPERATOR_OTF)
    plain_ms, plain_its = timed(one_by_one, reps=1)
    P.vie_destroy(h)
    # agreement of the lockstep solutions with the plain solves (last source)
    dif = float(np.linalg.norm(U_lock[-1] - u1.detach().cpu().numpy()) / np.linalg.norm(U_lock[-1]))
    return {"sources": nrhs, "medium": "2D heterogeneous 128x128 (the bench medium)",
            "assemble_bf16x3_ms": asm_ms,
            "lockstep_bf16x3_ms": lock_ms,
            "lockstep_bf16x3_iters_max": max(r["iters"] for r in reps),
            "lockstep_bf16x3_relres_max": max(r["relres"] for r in reps),
            "lockstep_learned_bf16x3_ms": lockl_ms,
            "lockstep_learned_iters_max": max(r["iters"] for r in repl),
            "lockstep_learned_relres_max": max(r["relres"] for r in repl),
            "single_bf16x3_gemv_ms": single_ms, "single_iters_max": max(single_its),
            "plain_on_the_fly_ms": plain_ms, "plain_iters_max": max(plain_its),
            "lockstep_vs_plain_rel_diff_last_source": dif}


def measure_batch(P, torch, stream, local, reps=3):
    """16 uneven 2D grids n = 64 ... 256 (Sum N^2 = 1.94e10 pairs) replayed from
    one CUDA graph, the persistent tile-pair launch's configuration autotuned:
    with the automatic kernel choice (the displacement kernel for n <= 258, one
    launch each, the persistent launch for the rest) and with every grid in the
    one persistent launch."""
    media = V.uneven_media()
    ns = [m.n for m in media]
    g = torch.as_tensor(np.concatenate([m.f for m in media]), dtype=torch.float64,
                        device=f"cuda:{local}")
    y = torch.empty_like(g)
    pairs = float(sum(m.N * m.N for m in media))
    out = {"grids": ns, "pairs": pairs}
    for name, kernel in (("auto", P.VIE_KERNEL_AUTO), ("persistent_only", P.VIE_KERNEL_SYMMETRIC)):
        b = P.vie_batch_create(ns, [m.sigma_t for m in media], [m.sigma_s for m in media], device=local,
                               kernel=kernel)
        t0 = time.perf_counter()
        cfg = P.vie_batch_autotune(b)
        tune_s = time.perf_counter() - t0
        P.vie_batch_apply(b, P.VIE_OP_K_SIGMA_S, g, y)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            P.vie_batch_apply(b, P.VIE_OP_K_SIGMA_S, g, y)
        e.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(e) / reps
        P.vie_batch_destroy(b)
        row = {"ms": ms, "gpair_per_s": pairs / (ms * 1e-3) / 1e9,
               "config": {"groups_per_cta": cfg[0], "smem_policy": cfg[1]}, "autotune_s": tune_s}
        if name == "auto":
            out.update(row)
        else:
            out[name] = row
    return out


def measure_learned(P, torch, local, seeds=(9004, 9005)):
    """Learned right preconditioner (4-level, 32-channel U-Net trained at 128^2
    by paper_1610_00835_gb300/train_unet.py) on held-out 256^2 strongly
    scattering media: FGMRES + network vs GMRES, both with the assembled BF16
    hi/lo operator, to 1e-6; assembly time reported separately."""
    weights = os.path.join(ROOT, "paper_1610_00835_gb300", "data", "unet_l4_c32.bin")
    net = P.vie_unet_create(4, 32, device=local)
    P.vie_unet_load(net, weights)
    rows = []
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for sd in seeds:
        m = V.diffusive_training_medium(256, sd)
        h = P.vie_create(2, 256, m.sigma_t, m.sigma_s, device=local)
        torch.cuda.synchronize()
        a.record()
        P.vie_assemble(h, P.VIE_OPERATOR_BF16X3)
        b.record()
        torch.cuda.synchronize()
        asm = a.elapsed_time(b)
        f = torch.as_tensor(m.f, dtype=torch.float64, device=f"cuda:{local}")
        U = torch.empty_like(f)
        row = {"seed": sd, "assemble_ms": asm}
        for name, pre in (("gmres", None), ("fgmres_learned", net), ("fgmres_fft", "fft"),
                          ("fgmres_diffusion", "diffusion")):
            if pre == "fft":
                P.vie_set_fft_preconditioner(h)
            elif pre == "diffusion":
                P.vie_set_diffusion_preconditioner(h)
            else:
                P.vie_set_preconditioner(h, pre, 5.0)
            P.vie_solve_gmres(h, f, U, rtol=RTOL, restart=128)
            torch.cuda.synchronize()
            a.record()
            rep = P.vie_solve_gmres(h, f, U, rtol=RTOL, restart=128)
            b.record()
            torch.cuda.synchronize()
            row[name] = {"iters": rep["iters"], "ms": a.elapsed_time(b), "relres": rep["relres"],
                         "fell_back": rep["fell_back"]}
        P.vie_set_fft_preconditioner(h, False)
        P.vie_set_diffusion_preconditioner(h, False)
        P.vie_destroy(h)
        rows.append(row)
    return {"grid": "256x256 (65536 unknowns), strongly scattering bump media, held out",
            "operator": "assembled BF16 hi/lo (17.2 GB)", "media": rows}


def measure_paper_preconditioners(P, torch, local):
    """The FFT and diffusion preconditioners (Section 4.4, Eqs. EQ: FFT, EQ:SOL
    FFT and EQ:DA) in the setting of the paper's Experiments V and VI on a
    128^2 grid: constant mu_a = 0.2 and mu_s = 10, 20, 40, 80, a Gaussian
    source at the centre.  GMRES(64) and FGMRES(64) with each preconditioner,
    on the fast FP32 path to 1e-6 and on FP64 pairs with the closed-form tau
    to 1e-10 (the FP32 tiles' rounding floors the residual near 1e-7); solve
    times by CUDA events after one warm-up solve, setups reported apart."""
    n = 128
    xs = V.cell_centres(2, n)
    f = torch.as_tensor(np.exp(-np.sum((xs - 0.5) ** 2, axis=1) / (2 * 0.1 ** 2)), dtype=torch.float64,
                        device=f"cuda:{local}")
    U = torch.empty_like(f)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows = []
    for path, kw, rtol in (("fp32_march", {}, RTOL),
                           ("fp64_closed", {"tau_mode": P.VIE_TAU_CLOSED, "precision": P.VIE_PREC_FP64}, 1e-10)):
        for mu_s in (10.0, 20.0, 40.0, 80.0):
            st, ss = np.full(n * n, mu_s + 0.2), np.full(n * n, mu_s)
            h = P.vie_create(2, n, st, ss, device=local, **kw)
            row = {"path": path, "mu_s": mu_s, "rtol": rtol}
            for name in ("gmres", "fgmres_fft", "fgmres_diffusion"):
                if name == "fgmres_fft":
                    t0 = time.perf_counter()
                    P.vie_set_fft_preconditioner(h)
                    row["fft_setup_ms"] = (time.perf_counter() - t0) * 1e3
                elif name == "fgmres_diffusion":
                    t0 = time.perf_counter()
                    P.vie_set_diffusion_preconditioner(h)
                    row["diffusion_setup_ms"] = (time.perf_counter() - t0) * 1e3
                P.vie_solve_gmres(h, f, U, rtol=rtol, maxit=3000)
                torch.cuda.synchronize()
                a.record()
                rep = P.vie_solve_gmres(h, f, U, rtol=rtol, maxit=3000)
                b.record()
                torch.cuda.synchronize()
                row[name] = {"iters": rep["iters"], "ms": a.elapsed_time(b), "relres": rep["relres"],
                             "fell_back": rep["fell_back"]}
            P.vie_destroy(h)
            rows.append(row)
    return {"grid": "128x128, constant mu_a = 0.2 and mu_s (Experiments V and VI of the paper at h = 1/128)",
            "paper": "h = 1/512, FMM operator, tol 1e-12, mu_s = 10/20/40/80: Table TAB:EXP VI FFT-preconditioned "
                     "9/11/13/15 vs 21/34/78/110 iterations; Table TAB:EXP V diffusion-preconditioned 36/38/42/52",
            "rows": rows}


def measure_paper_fmm_tables(P, torch, local):
    """The paper's Experiments I and II (Tables TAB:Con Coeff and TAB:Var Coeff)
    with the FMM operator (Section 3.3): homogeneous mu_s = 2.0, mu_a = 0.2 with
    the closed-form tau (the paper evaluates E analytically there), and the
    medium of Eq. EQ:Coeff (mu_a = 0.2, mu_s = 3 + 2 exp(-|x - (1/2, 1/2)|^2 / 4))
    with the 64-step march; N = 32^2 .. 512^2, Chebyshev orders 4, 6, 9.  The
    paper's ring source exists only as a figure; a ring of radius 0.25 and
    width 0.05 about the centre stands in.  Per case: assembly (the paper's
    T^fmm: every kernel value computed and cached), the GMRES(64) solve to 1e-6
    and its time per operator apply (T_g^fmm), and E_l2 = ||U_fmm - U_dir|| /
    ||U_dir|| against the on-the-fly direct solve up to 256^2 (the paper's
    direct path stopped at 128^2)."""
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = []
    for medium in ("homogeneous", "eq_coeff"):
        for n in (32, 64, 128, 256, 512):
            xs = V.cell_centres(2, n)
            r = np.sqrt(np.sum((xs - 0.5) ** 2, axis=1))
            f = torch.as_tensor(np.exp(-(r - 0.25) ** 2 / (2 * 0.05 ** 2)), dtype=torch.float64,
                                device=f"cuda:{local}")
            if medium == "homogeneous":
                ss = np.full(n * n, 2.0)
                kw = {"tau_mode": P.VIE_TAU_CLOSED}
            else:
                ss = 3.0 + 2.0 * np.exp(-r ** 2 / 4.0)
                kw = {}
            st = ss + 0.2
            h = P.vie_create(2, n, st, ss, device=local, **kw)
            U = torch.empty_like(f)
            U_dir = None
            if n <= 256:
                P.vie_solve_gmres(h, f, U, rtol=RTOL)
                U_dir = U.clone()
            for order in (4, 6, 9):
                torch.cuda.synchronize()
                a.record()
                P.vie_assemble_fmm(h, order)
                b.record()
                torch.cuda.synchronize()
                asm = a.elapsed_time(b)
                P.vie_solve_gmres(h, f, U, rtol=RTOL)
                torch.cuda.synchronize()
                a.record()
                rep = P.vie_solve_gmres(h, f, U, rtol=RTOL)
                b.record()
                torch.cuda.synchronize()
                ms = a.elapsed_time(b)
                row = {"medium": medium, "N": n * n, "order": order, "assemble_ms": asm, "solve_ms": ms,
                       "iters": rep["iters"], "ms_per_apply": ms / max(1, rep["n_apply"])}
                if U_dir is not None:
                    row["E_l2_vs_direct"] = float(torch.linalg.norm(U - U_dir) / torch.linalg.norm(U_dir))
                out.append(row)
            P.vie_destroy(h)
    return {"rtol": RTOL, "source": "ring stand-in (radius 0.25, width 0.05)",
            "paper": "MATLAB on one i7-6560U core, tol 1e-12: order 6, N = 262144: T^fmm 13.9 s (homogeneous) / "
                     "T_g^fmm 0.27 s per iteration; order 4 heterogeneous T^fmm 114 s; E_l2 1.3e-6 (homogeneous, "
                     "order 6), 2.0e-4 .. 3.5e-4 (heterogeneous, order 4)",
            "rows": out}


def measure_other_configs(P, torch, local, reps=3):
    """The two other single-GPU workloads of the method: the homogeneous 32^2
    medium in FP64 with the closed-form tau (GMRES to 1e-10), and the 32^3
    heterogeneous medium (FP32 tiles, S = 64): one apply, the GMRES solve to
    1e-6 (on the fly, and on K assembled from the pair weights), and the
    step-two sweep on 128 Fibonacci directions (Algorithm 1, S.3).  Median of `reps` runs after one warm-up, CUDA events."""
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            a.record()
            out = fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts), out

    dev = f"cuda:{local}"
    m1 = V.homogeneous_medium(2, 32, 1.1, 1.0)
    h1 = P.vie_create(2, 32, m1.sigma_t, m1.sigma_s, tau_mode=P.VIE_TAU_CLOSED, precision=P.VIE_PREC_FP64,
                      device=local)
    f1 = torch.as_tensor(m1.f, dtype=torch.float64, device=dev)
    U1 = torch.empty_like(f1)
    ms1, rep1 = timed(lambda: P.vie_solve_gmres(h1, f1, U1, rtol=1e-10))
    P.vie_destroy(h1)
    m3 = V.heterogeneous_3d(n=32)
    h3 = P.vie_create(3, 32, m3.sigma_t, m3.sigma_s, device=local)
    f3 = torch.as_tensor(m3.f, dtype=torch.float64, device=dev)
    U3 = torch.empty_like(f3)
    y3 = torch.empty_like(f3)
    ms_apply, _ = timed(lambda: P.vie_apply(h3, P.VIE_OP_K_SIGMA_S, f3, y3, 1))
    work3 = P.vie_get_kernel_work(h3)   # multiply-adds of the tau sums per apply
    ms3, rep3 = timed(lambda: P.vie_solve_gmres(h3, f3, U3, rtol=RTOL))
    M = 128
    dirs = torch.as_tensor(V.fibonacci_directions(M).astype(np.float32), device=dev)  # [M, 3]
    Phi = torch.empty(M * m3.N, dtype=torch.float32, device=dev)
    ms_sweep, _ = timed(lambda: P.ert_sweep(h3, U3, f3, dirs, Phi))
    # the chosen solver: K assembled from the 3D displacement kernel's pair
    # weights (each unordered pair marched once), then GMRES on the GEMV
    asm3, _ = timed(lambda: P.vie_assemble(h3, P.VIE_OPERATOR_FP32))
    U3c = torch.empty_like(f3)
    ms3c, rep3c = timed(lambda: P.vie_solve_gmres(h3, f3, U3c, rtol=RTOL))
    dif3 = float(torch.linalg.norm(U3c - U3) / torch.linalg.norm(U3))
    P.vie_assemble(h3, P.VIE_OPERATOR_OTF)
    P.vie_destroy(h3)
    return {"homogeneous_32x32_fp64": {"tau": "closed form", "rtol": 1e-10, "solve_ms": ms1,
                                       "iters": rep1["iters"], "relres": rep1["relres"]},
            "heterogeneous_32x32x32": {"N": m3.N, "apply_ms": ms_apply,
                                       "apply_gpair_per_s": float(m3.N) * m3.N / ms_apply / 1e6,
                                       "tau_multiply_adds": work3,
                                       "apply_tflops": 2.0 * work3 / ms_apply / 1e9,
                                       "solve_ms": ms3, "iters": rep3["iters"], "relres": rep3["relres"],
                                       "chosen": {"solver": "assembled FP32 K from the 3D displacement kernel's "
                                                            "pair weights (4.3 GB) + FP64 GMRES(64)",
                                                  "assemble_ms": asm3, "solve_ms": ms3c,
                                                  "total_ms": asm3 + ms3c, "iters": rep3c["iters"],
                                                  "relres": rep3c["relres"], "rel_diff_vs_plain": dif3},
                                       "sweep_directions": M, "sweep_ms": ms_sweep,
                                       "sweep_rays_per_s": M * m3.N / ms_sweep * 1e3}}


def reduce_over_ranks(dist, total_ms: float, pairs: float, device) -> tuple:
    """Whole-job aggregation over the ranks: the slowest rank's time and the
    pairs all ranks processed (each rank solves its own medium)."""
    if dist is None:
        return total_ms, pairs
    import torch
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([pairs], dtype=torch.float64, device=device)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p.item())


def run_ours(args):
    import torch
    import paper_1610_00835_gb300 as P

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    P.load()
    m = medium(rank)
    N = m.N
    # the first handle of a grid size in a process builds the displacement
    # stencils and work list on the host (shared by later handles of that size)
    t0 = time.perf_counter()
    h = P.vie_create(2, m.n, m.sigma_t, m.sigma_s, steps=S_STEPS, device=local)
    torch.cuda.synchronize()
    first_create_ms = {f"{m.n}x{m.n}": (time.perf_counter() - t0) * 1e3}
    # the same for 256^2, before any later leg has built that size
    m256 = V.heterogeneous_2d(n=256)
    t0 = time.perf_counter()
    h256 = P.vie_create(2, 256, m256.sigma_t, m256.sigma_s, steps=S_STEPS, device=local)
    torch.cuda.synchronize()
    first_create_ms["256x256"] = (time.perf_counter() - t0) * 1e3
    P.vie_destroy(h256)
    f_dev = torch.as_tensor(m.f, dtype=torch.float64, device=f"cuda:{local}")
    U = torch.empty(N, dtype=torch.float64, device=f"cuda:{local}")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=f"cuda:{local}")  # 256 MB > L2
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        P.vie_solve_gmres(h, f_dev, U, rtol=RTOL)
    torch.cuda.synchronize()
    U_or = oracle_solution(rank)
    launches0 = P.vie_kernel_launches()
    step_ms, reps = [], []
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush_l2(flush)
            torch.cuda.synchronize()
            barrier()
            nvtx_push(torch, "timed_step")
            start.record(stream)
            rep = P.vie_solve_gmres(h, f_dev, U, rtol=RTOL, time_apply=True)
            stop.record(stream)
            torch.cuda.synchronize()
            nvtx_pop(torch)
            step_ms.append(start.elapsed_time(stop))
            reps.append(rep)
    launches = P.vie_kernel_launches() - launches0
    err_plain = err_vs_oracle(U, U_or)
    total_ms = sum(step_ms)
    pairs = sum(r["n_apply"] for r in reps) * float(N) * N
    total_ms, pairs = reduce_over_ranks(dist, total_ms, pairs, f"cuda:{local}")
    value = pairs / (total_ms * 1e-3) / 1e9

    # roofline of the pair kernel, from the per-launch CUDA events of the timed steps
    n_apply = sum(r["n_apply"] for r in reps)
    kern_ms = sum(r["t_apply_kernel_ms"] for r in reps) / n_apply
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    clocks = clk.summary()
    max_mhz = clocks["sm_max_mhz"] or 2070.0
    kernel = P.vie_get_kernel(h)
    fma = P.vie_get_kernel_work(h)                                 # multiply-adds per apply
    peak = sms * 128 * 2 * max_mhz * 1e6 / 1e12                    # FP32 TFLOP/s at max clock
    achieved = 2.0 * fma / (kern_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": PAIR_KERNEL_DRAM_BYTES.get(kernel),
                "resource": "FP32 FMA pipe (the kernel is issue-bound: loads and bookkeeping share the issue slots)",
                "kernel": KERNEL_NAMES.get(kernel, str(kernel)), "kernel_ms": kern_ms,
                "work": f"{fma:.4g} multiply-adds per apply (tau sums, the method's own count), 2 FLOP each",
                "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 FLOP x {max_mhz:.0f} MHz (max clock)",
                "gpair_per_s_apply": float(N) * N / (kern_ms * 1e-3) / 1e9}
    if clocks["sm_mhz"]:
        roofline["frac_at_measured_clock"] = achieved / (sms * 128 * 2 * clocks["sm_mhz"] * 1e6 / 1e12)
    # the per-pair work of the per-sample march (about 13 S + 12 FP32 issues per
    # ordered pair at S = 64: 844), against the FP32 issue rate of the part: the
    # stencil form does far fewer issues per pair, so this reads above 1
    per_pair = 13 * S_STEPS + 12
    issue_rate = sms * 128 * max_mhz * 1e6
    roofline["per_sample_march_basis"] = {
        "fp32_issues_per_pair": per_pair,
        "pair_bound_gpair_per_s": issue_rate / per_pair / 1e9,
        "frac": float(N) * N / (kern_ms * 1e-3) / (issue_rate / per_pair),
        "note": "ordered pairs N^2 per apply; above 1 because the stencil march groups the samples "
                "by lattice cell (about 142 multiply-adds per pair at 128^2, symmetric pairs once)"}

    chosen = measure_assembled(P, torch, h, f_dev, U, flush, stream, args, P.VIE_OPERATOR_SYM32, U_or)
    asm_bf16 = measure_assembled(P, torch, h, f_dev, U, flush, stream, args, P.VIE_OPERATOR_BF16X3, U_or)
    asm_pairs = measure_assembled(P, torch, h, f_dev, U, flush, stream, args, P.VIE_OPERATOR_PAIRS32, U_or)
    asm_fp32 = measure_assembled(P, torch, h, f_dev, U, flush, stream, args, P.VIE_OPERATOR_FP32, U_or)
    net = P.vie_unet_create(4, 32, device=local)
    P.vie_unet_load(net, os.path.join(ROOT, "paper_1610_00835_gb300", "data", "unet_l4_c32.bin"))
    learned_128 = measure_assembled(P, torch, h, f_dev, U, flush, stream, args, P.VIE_OPERATOR_SYM32,
                                    U_or, net=net)
    P.vie_unet_destroy(net)
    chosen_fft = measure_assembled(P, torch, h, f_dev, U, flush, stream, args, P.VIE_OPERATOR_SYM32, U_or,
                                   fft=True)
    chosen_fmm = measure_assembled(P, torch, h, f_dev, U, flush, stream, args, P.VIE_OPERATOR_FMM, U_or)
    mii = measure_mii(P, torch, m, f_dev, flush, stream, args, local, rank, U_or)
    product = measure_bf16x3_product(P, torch, m, h, stream, args, local)
    multi = measure_multi_source(P, torch, m, stream, local)
    batch = measure_batch(P, torch, stream, local)
    others = measure_other_configs(P, torch, local)
    learned = measure_learned(P, torch, local)
    paper_pre = measure_paper_preconditioners(P, torch, local)
    paper_fmm = measure_paper_fmm_tables(P, torch, local)

    # end to end through the C ABI from host buffers
    e2e_steps = max(1, min(args.steps, 10))
    U_host = np.zeros(N)
    t_e2e = []
    for _ in range(e2e_steps):
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        he = P.vie_create(2, m.n, m.sigma_t, m.sigma_s, steps=S_STEPS, device=local)
        rep_e = P.vie_solve_gmres(he, m.f, U_host, rtol=RTOL)
        P.vie_destroy(he)
        t_e2e.append(time.perf_counter() - t0)
    e2e_pairs = rep_e["n_apply"] * float(N) * N * e2e_steps
    e2e = {"value": e2e_pairs / sum(t_e2e) / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": 3 * N * 8, "d2h_bytes_per_step": N * 8,
           "note": "each step creates its handle; the stencil geometry of the grid size is built by "
                   "the first handle in the process and reused (first_create_ms)",
           "first_create_ms": first_create_ms}

    line = None
    if rank == 0:
        cpu = cpu_baseline_sample(m) if world == 1 else None
        last = reps[-1]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "ms_per_step_median": statistics.median(step_ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 tiles / f64 krylov",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "S": S_STEPS, "rtol": RTOL,
                       "solver": "plain: FP64 GMRES(64), on-the-fly FP32 operator",
                       "parallelism": f"replicas x{world}",
                       "l2": "flushed between steps (256 MB write)"},
            "solve": {"iters": last["iters"], "n_apply": last["n_apply"],
                      "relres": last["relres"], "solve_ms_plain": total_ms / args.steps,
                      "apply_ms": sum(r["t_apply_ms"] for r in reps) / n_apply,
                      "err_vs_oracle": err_plain,
                      "solve_ms_chosen": chosen["solve_ms"], "chosen": chosen,
                      "assembled_bf16x3": asm_bf16, "assembled_pairs32": asm_pairs, "assembled_fp32": asm_fp32,
                      "chosen_learned": learned_128,
                      "chosen_fft": chosen_fft,
                      "chosen_fmm": chosen_fmm,
                      "m_ii": mii,
                      "oracle_U": "tests/golden/bench_U_2d_128.npy (FP64 oracle, rtol 1e-11)"
                      if U_or is not None else None},
            "bf16x3_product": product,
            "multi_source_solve": multi,
            "batch_uneven_grids": batch,
            "learned_preconditioner": learned,
            "paper_preconditioners": paper_pre,
            "paper_fmm_tables": paper_fmm,
            "other_workloads": others,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": int(launches),
        }
        print(json.dumps(line), flush=True)
    P.vie_destroy(h)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_only(args):
    """One workload alone, repeated (a small driver for profilers): the step-two
    sweep of the 32^3 medium on 128 directions, the 16-grid batched apply, or the
    learned preconditioner's forward pass at 256^2."""
    import torch
    import paper_1610_00835_gb300 as P

    dev = "cuda:0"
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.only == "sweep":
        m = V.heterogeneous_3d(n=32)
        h = P.vie_create(3, 32, m.sigma_t, m.sigma_s)
        f = torch.as_tensor(m.f, dtype=torch.float64, device=dev)
        U = torch.empty_like(f)
        P.vie_solve_gmres(h, f, U, rtol=RTOL)
        dirs = torch.as_tensor(V.fibonacci_directions(128).astype(np.float32), device=dev)
        Phi = torch.empty(128 * m.N, dtype=torch.float32, device=dev)
        run = lambda: P.ert_sweep(h, U, f, dirs, Phi)  # noqa: E731
    elif args.only == "batch":
        media = [m for m in V.uneven_media() if m.n <= args.n]   # --n: the largest grid taken
        b = P.vie_batch_create([m.n for m in media], [m.sigma_t for m in media], [m.sigma_s for m in media],
                               kernel=P.VIE_KERNEL_SYMMETRIC)
        g = torch.as_tensor(np.concatenate([m.f for m in media]), dtype=torch.float64, device=dev)
        y = torch.empty_like(g)
        run = lambda: P.vie_batch_apply(b, P.VIE_OP_K_SIGMA_S, g, y)  # noqa: E731
    elif args.only == "train":
        # one training step of the U-Net (FP32 forward, backward, Adam) on random images
        net = P.vie_unet_create(4, 32)
        n, B = args.unet_n, args.batch
        x = torch.randn(B * 3 * n * n, dtype=torch.float32, device=dev)
        t = torch.randn(B * n * n, dtype=torch.float32, device=dev)
        run = lambda: P.vie_unet_train_step(net, x, t, B, n, 1e-4)  # noqa: E731
    else:
        net = P.vie_unet_create(4, 32)
        P.vie_unet_load(net, os.path.join(ROOT, "paper_1610_00835_gb300", "data", "unet_l4_c32.bin"))
        n, B = args.unet_n, args.batch
        x = torch.randn(B * 3 * n * n, dtype=torch.float32, device=dev)
        o = torch.empty(B * n * n, dtype=torch.float32, device=dev)
        run = lambda: P.vie_unet_forward(net, x, o, B, n, use_bf16=True)  # noqa: E731
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    a.record()
    for _ in range(args.steps):
        run()
    e.record()
    torch.cuda.synchronize()
    print(json.dumps({"mode": "only", "workload": args.only, "ms": a.elapsed_time(e) / args.steps}), flush=True)
    return 0


def run_apply_only(args):
    """K operator applies on the bench medium (a small driver for profilers)."""
    import torch
    import paper_1610_00835_gb300 as P

    m = V.heterogeneous_2d(n=args.n) if args.dim == 2 else V.heterogeneous_3d(n=args.n)
    h = P.vie_create(args.dim, m.n, m.sigma_t, m.sigma_s, steps=S_STEPS,
                     disc=P.VIE_DISC_MII if args.disc == "m2" else P.VIE_DISC_MIII)
    mode = {"otf": P.VIE_OPERATOR_OTF, "fp32": P.VIE_OPERATOR_FP32, "bf16x3": P.VIE_OPERATOR_BF16X3,
            "pairs32": P.VIE_OPERATOR_PAIRS32, "sym32": P.VIE_OPERATOR_SYM32, "fmm": P.VIE_OPERATOR_FMM}[args.operator]
    P.vie_assemble(h, mode)
    nrhs = args.nrhs
    G = V.bump_sources(args.dim, m.n, nrhs, seed=V.seed_for(4)) if nrhs > 1 else m.f[None, :]
    g = torch.as_tensor(G.ravel(), dtype=torch.float64, device="cuda:0")
    y = torch.empty_like(g)
    for _ in range(args.warmup):
        P.vie_apply(h, P.VIE_OP_K_SIGMA_S, g, y, nrhs)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        P.vie_apply(h, P.VIE_OP_K_SIGMA_S, g, y, nrhs)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    print(json.dumps({"mode": "apply-only", "operator": args.operator, "disc": args.disc, "nrhs": nrhs,
                      "dim": args.dim, "n": m.n, "N": m.N, "ms_per_apply": ms,
                      "gpair_per_s": float(m.N) * m.N * nrhs / ms / 1e6}), flush=True)
    P.vie_destroy(h)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--apply-only", action="store_true",
                    help="time operator applies only (profiling driver)")
    ap.add_argument("--dim", type=int, default=2)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--operator", choices=["otf", "fp32", "bf16x3", "pairs32", "sym32", "fmm"], default="otf")
    ap.add_argument("--unet-n", type=int, default=256, help="--only unet / train: grid of the images")
    ap.add_argument("--batch", type=int, default=1, help="--only unet / train: images per forward")
    ap.add_argument("--only", choices=["sweep", "batch", "unet", "train"], default=None,
                    help="run one workload alone, for profilers")
    ap.add_argument("--disc", choices=["m3", "m2"], default="m3",
                    help="apply-only: discretisation M-iii (default) or M-ii (2D)")
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.apply_only:
        return run_apply_only(args)
    if args.only:
        return run_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
