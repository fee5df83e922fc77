"""Write the FP64 oracle solution of the benchmark medium (test infrastructure).

The benchmark solves the 2D heterogeneous 128x128 medium of seed 2000
(sigma_t = 1 + 4 seeded bumps, sigma_s = 0.9 sigma_t, Gaussian source f at
the centre, S = 64 march): phi = A f, then (I - K) U = phi (Algorithm 1,
S.1-S.2).  This script calls only the FP64 CPU oracle and the seeded input
generators; it writes bench_U_2d_128.npy (U, FP64 [16384]) and
bench_U_2d_128.json (how it was made).  It takes about ten minutes on 8 cores.
With --mii it solves the same medium discretised by approach M-ii (Section
3.2, Remark REM: NEW KERNEL) and writes bench_U_2d_128_mii.{npy,json}.

Usage: python tests/golden/make_bench_solution.py [--mii]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import vie_synth as V  # noqa: E402

SEED = V.seed_for(2, 0)
RTOL = 1e-11


def main():
    mii = "--mii" in sys.argv[1:]
    mode = O.TAU_MARCH | (O.DISC_MII if mii else 0)
    stem = "bench_U_2d_128_mii" if mii else "bench_U_2d_128"
    m = V.heterogeneous_2d(n=128, seed=SEED)
    t0 = time.time()
    phi = O.apply(2, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW, mode=mode)
    U, iters, relres, ok = O.gmres(2, m.sigma_t, m.sigma_s, phi, rtol=RTOL, mode=mode)
    if not ok:
        raise SystemExit(f"oracle GMRES did not converge: relres {relres}")
    np.save(os.path.join(HERE, stem + ".npy"), U)
    with open(os.path.join(HERE, stem + ".json"), "w") as fh:
        json.dump({"what": "FP64 oracle solution U of (I - K) U = A f, Algorithm 1 S.1-S.2",
                   "discretisation": "M-ii (Remark REM: NEW KERNEL)" if mii else "M-iii",
                   "medium": "vie_synth.heterogeneous_2d(n=128, seed=2000)", "S": 64,
                   "solver": "oracle GMRES(64), x0 = 0", "rtol": RTOL, "iters": iters,
                   "relres": relres, "seconds": round(time.time() - t0, 1),
                   "threads": O.num_threads()}, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
