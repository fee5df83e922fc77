"""Seeded synthetic inputs: media, sources and direction sets.

This module is shared by the CUDA path's tests and benchmarks and by the FP64
oracle.  It holds no arithmetic of the method itself (no kernel, no line
integral, no quadrature): it only draws the coefficient fields sigma_t,
sigma_s, the source f and the unit direction sets that both sides consume.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out here from its
published definition so that every medium is reproducible from its seed on
any machine.

Grid convention (Section 3.1, uniform grid of cell size h on the unit square
or cube): n cells per side, N = n**d unknowns, h = 1/n, cell centres at
x = (i + 1/2) h, linear index j = ix + n*iy (+ n*n*iz), x fastest.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream; ``uniform()`` returns doubles in [0, 1)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))


def seed_for(config: int, item: int = 0) -> int:
    """Seed of item ``item`` of workload ``config`` (1000*config + item)."""
    return 1000 * config + item


def cell_centres(dim: int, n: int) -> np.ndarray:
    """Cell-centre coordinates, shape [N, dim], index j = ix + n*iy (+ n^2*iz)."""
    c = (np.arange(n, dtype=np.float64) + 0.5) / n
    if dim == 2:
        yy, xx = np.meshgrid(c, c, indexing="ij")
        return np.stack([xx.ravel(), yy.ravel()], axis=1)
    if dim == 3:
        zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
        return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    raise ValueError("dim must be 2 or 3")


@dataclass
class Bump:
    amp: float
    width: float
    centre: tuple


def draw_bumps(rng: SplitMix64, dim: int, count: int, amp=(0.5, 3.0),
               width=(0.05, 0.2), centre=(0.2, 0.8)) -> list:
    out = []
    for _ in range(count):
        a = rng.uniform(*amp) if isinstance(amp, tuple) else float(amp)
        w = rng.uniform(*width)
        c = tuple(rng.uniform(*centre) for _ in range(dim))
        out.append(Bump(a, w, c))
    return out


def bump_field(dim: int, n: int, bumps, base: float = 0.0) -> np.ndarray:
    """base + sum_b a_b exp(-|x - c_b|^2 / (2 w_b^2)) sampled at cell centres."""
    x = cell_centres(dim, n)
    v = np.full(x.shape[0], base, dtype=np.float64)
    for b in bumps:
        d2 = np.sum((x - np.asarray(b.centre)) ** 2, axis=1)
        v += b.amp * np.exp(-d2 / (2.0 * b.width ** 2))
    return v


def gaussian_source(dim: int, n: int, centre=None, width: float = 0.1) -> np.ndarray:
    if centre is None:
        centre = (0.5,) * dim
    return bump_field(dim, n, [Bump(1.0, width, tuple(centre))])


@dataclass
class Medium:
    dim: int
    n: int
    sigma_t: np.ndarray
    sigma_s: np.ndarray
    f: np.ndarray
    homogeneous: bool = False
    label: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.n ** self.dim

    @property
    def h(self) -> float:
        return 1.0 / self.n


def homogeneous_medium(dim=2, n=32, sigma_t=1.1, sigma_s=1.0, width=0.1) -> Medium:
    """2D homogeneous square, constant coefficients, Gaussian source at the centre."""
    N = n ** dim
    return Medium(dim, n, np.full(N, sigma_t), np.full(N, sigma_s),
                  gaussian_source(dim, n, width=width), True,
                  f"homogeneous {n}^{dim} sigma_t={sigma_t} sigma_s={sigma_s}")


def bump_medium(dim: int, n: int, nbumps: int, ratio: float, seed: int,
                width_src: float = 0.1) -> Medium:
    """sigma_t = 1 + sum of seeded Gaussian bumps, sigma_s = ratio * sigma_t."""
    rng = SplitMix64(seed)
    bumps = draw_bumps(rng, dim, nbumps)
    st = bump_field(dim, n, bumps, base=1.0)
    return Medium(dim, n, st, ratio * st, gaussian_source(dim, n, width=width_src),
                  False, f"bumps {n}^{dim} x{nbumps} seed={seed}",
                  {"bumps": bumps, "seed": seed})


def heterogeneous_2d(n: int = 128, seed: int = seed_for(2)) -> Medium:
    """128^2 medium: 1 + 4 bumps (amp U[0.5,3], width U[0.05,0.2]), sigma_s = 0.9 sigma_t."""
    return bump_medium(2, n, 4, 0.9, seed)


def heterogeneous_3d(n: int = 32, seed: int = seed_for(3)) -> Medium:
    """32^3 medium: 1 + 6 bumps, sigma_s = 0.8 sigma_t."""
    return bump_medium(3, n, 6, 0.8, seed)


def bump_sources(dim: int, n: int, count: int, seed: int) -> np.ndarray:
    """[count, N] seeded Gaussian bump sources (amp 1, width U[0.05,0.2], centre U[0.2,0.8]^d)."""
    rng = SplitMix64(seed)
    bumps = draw_bumps(rng, dim, count, amp=1.0)
    return np.stack([bump_field(dim, n, [b]) for b in bumps])


def uneven_grid_sizes(count: int = 16, lo: int = 64, hi: int = 256) -> list:
    """n_i = lo + round((hi - lo) * i / (count - 1)), i = 0..count-1."""
    if count == 1:
        return [lo]
    return [lo + int(math.floor((hi - lo) * i / (count - 1) + 0.5)) for i in range(count)]


def uneven_media(count: int = 16, seed0: int = seed_for(4, 100)) -> list:
    return [bump_medium(2, n, 4, 0.9, seed0 + i) for i, n in enumerate(uneven_grid_sizes(count))]


def random_training_medium(n: int, seed: int) -> Medium:
    """Random bump medium for learned-preconditioner data: 2..6 bumps, ratio U[0.5, 0.95]."""
    rng = SplitMix64(seed)
    nb = 2 + int(rng.uniform() * 5)
    ratio = rng.uniform(0.5, 0.95)
    bumps = draw_bumps(rng, 2, nb)
    st = bump_field(2, n, bumps, base=1.0)
    srcb = draw_bumps(rng, 2, 1 + int(rng.uniform() * 3), amp=(0.5, 1.5))
    f = bump_field(2, n, srcb)
    return Medium(2, n, st, ratio * st, f, False, f"train {n}^2 seed={seed}",
                  {"seed": seed, "ratio": ratio})


def diffusive_training_medium(n: int, seed: int) -> Medium:
    """Strongly scattering bump medium (the regime of the paper's
    preconditioning experiments, mu_a small against mu_s): sigma_s = s (1 +
    sum of 1..4 bumps, amplitude U[0.2, 1], width U[0.05, 0.2]), s
    log-uniform in [4, 16]; sigma_t = sigma_s + mu_a, mu_a ~ U[0.1, 0.5]."""
    rng = SplitMix64(seed)
    nb = 1 + int(rng.uniform() * 4)
    s = math.exp(rng.uniform(math.log(4.0), math.log(16.0)))
    mu_a = rng.uniform(0.1, 0.5)
    bumps = draw_bumps(rng, 2, nb, amp=(0.2, 1.0))
    ss = s * bump_field(2, n, bumps, base=1.0)
    srcb = draw_bumps(rng, 2, 1 + int(rng.uniform() * 3), amp=(0.5, 1.5))
    f = bump_field(2, n, srcb)
    return Medium(2, n, ss + mu_a, ss, f, False, f"diffusive {n}^2 seed={seed}",
                  {"seed": seed, "s": s, "mu_a": mu_a})


def random_rhs(n: int, seed: int) -> np.ndarray:
    """A smooth right-hand side for (I - K) U = b: 2..5 Gaussian bumps with
    amplitudes U[-1, 1], widths U[0.03, 0.3], centres U[0.1, 0.9]^2."""
    rng = SplitMix64(seed)
    nb = 2 + int(rng.uniform() * 4)
    bumps = draw_bumps(rng, 2, nb, amp=(-1.0, 1.0), width=(0.03, 0.3), centre=(0.1, 0.9))
    return bump_field(2, n, bumps)


def random_field(n: int, seed: int, width=(0.05, 0.3), count=(4, 16)) -> np.ndarray:
    """A random field on the n x n centres: count[0]..count[1] Gaussian bumps,
    amplitudes U[-1, 1], widths U[width], centres U[0, 1]^2."""
    rng = SplitMix64(seed)
    nb = count[0] + int(rng.uniform() * (count[1] - count[0] + 1))
    bumps = draw_bumps(rng, 2, nb, amp=(-1.0, 1.0), width=width, centre=(0.0, 1.0))
    return bump_field(2, n, bumps)


def fibonacci_directions(M: int) -> np.ndarray:
    """[M, 3] unit vectors: z_m = 1 - (2m+1)/M, azimuth m * pi * (3 - sqrt 5)."""
    m = np.arange(M, dtype=np.float64)
    z = 1.0 - (2.0 * m + 1.0) / M
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = m * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def circle_directions(M: int) -> np.ndarray:
    """[M, 2] unit vectors at angles 2*pi*(m + 1/2)/M."""
    t = 2.0 * math.pi * (np.arange(M, dtype=np.float64) + 0.5) / M
    return np.stack([np.cos(t), np.sin(t)], axis=1)


def directions(dim: int, M: int) -> np.ndarray:
    return circle_directions(M) if dim == 2 else fibonacci_directions(M)


def linear_field(dim: int, n: int, alpha: float, beta) -> np.ndarray:
    """alpha + beta . x at cell centres (used for analytic line-integral checks)."""
    return alpha + cell_centres(dim, n) @ np.asarray(beta, dtype=np.float64)
