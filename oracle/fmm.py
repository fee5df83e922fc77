"""Interpolation-based FMM of Section 3.3 (Eqs. EQ: CHEB, EQ:Kernel Approx,
EQ: SUMMATION, EQ: M2L, EQ: L2L), 2D, FP64 numpy reference (TEST
INFRASTRUCTURE ONLY: imported by tests/ and nothing else).

It evaluates y = A s for the M-iii matrix A (Section 3.2) with the far field
replaced by Chebyshev interpolation of the kernel
    K(x, y) = h^2 exp(-tau(x, y)) / (2 pi |x - y|),
tau the S-step midpoint march of the bilinear sigma_t (clamped to the hull of
the cell centres), in the multilevel form of the Fong-Darve method:
    tree      : the n x n grid as a quadtree; leaves of b x b cells with
                n = 2^L b, b >= 8 and as small as the factors of two allow;
                level l has 2^l x 2^l boxes;
    S_p       : Eq. EQ: CHEB, the product over the axes of
                1/p + (2/p) sum_{k=1}^{p-1} T_k(u) T_k(v), u, v in [-1, 1];
                nodes: first-kind Chebyshev points cos((2i - 1) pi / (2p)),
                mapped affinely into each box (tensor product, m = mx + p my);
    near      : leaves B, C with |B - C| <= 1 in both box coordinates: the
                entries A_jk themselves (the self cell on the diagonal);
    far       : at each level l >= 2, box B and the boxes C of its
                interaction list (children of the neighbours of B's parent,
                not neighbours of B): L_B += K(nodes_B, nodes_C) W_C;
    upward    : W_leaf[m] = sum_{k in leaf} S_p(R^{-1} x_k, z_m) s_k (Eq.
                EQ: SUMMATION step 1), W_parent[m] = sum over the children and
                their nodes of S_p(R_parent^{-1} node', z_m) W_child[node'];
    downward  : L_child[m'] += sum_m S_p(R_parent^{-1} node'_m', z_m)
                L_parent[m]; y_j += sum_m S_p(R_leaf^{-1} x_j, z_m) L_leaf[m]
                (Eq. EQ: L2L).
"""
from __future__ import annotations

import math

import numpy as np

from . import selfcell


def leaf_levels(n: int):
    """(L, b): the number of levels below the root and the leaf side in cells."""
    L = 0
    while n % (2 ** (L + 1)) == 0 and n // 2 ** (L + 1) >= 8:
        L += 1
    return L, n // 2 ** L


def cheb_points(p: int) -> np.ndarray:
    return np.cos((2 * np.arange(1, p + 1) - 1) * np.pi / (2 * p))


def s1(p: int, u, v) -> np.ndarray:
    """The 1D factor of S_p (Eq. EQ: CHEB) for all pairs: [len(u), len(v)]."""
    u = np.clip(np.asarray(u, dtype=np.float64), -1.0, 1.0)
    v = np.asarray(v, dtype=np.float64)
    tu = np.arccos(u)[:, None] * np.arange(1, p)[None, :]
    tv = np.arccos(v)[:, None] * np.arange(1, p)[None, :]
    return 1.0 / p + (2.0 / p) * np.cos(tu) @ np.cos(tv).T


def interp_matrix(p: int, pts, lo, width) -> np.ndarray:
    """S_p(R^{-1} x, z_m) for points pts [k, 2] in the box [lo, lo + width]^2:
    [p^2, k], node m = mx + p my."""
    z = cheb_points(p)
    u = 2.0 * (np.asarray(pts)[:, 0] - lo[0]) / width - 1.0
    v = 2.0 * (np.asarray(pts)[:, 1] - lo[1]) / width - 1.0
    sx = s1(p, u, z)  # [k, p]
    sy = s1(p, v, z)
    return np.einsum("kb,ka->bak", sy, sx).reshape(p * p, -1)


def box_nodes(p: int, lo, width) -> np.ndarray:
    z = cheb_points(p)
    x = lo[0] + 0.5 * width * (z + 1.0)
    y = lo[1] + 0.5 * width * (z + 1.0)
    X, Y = np.meshgrid(x, y)  # [my, mx]
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def bilinear(sigma, n, px, py):
    """sigma~ at physical points (arrays), clamped to the hull of the centres."""
    S = np.asarray(sigma, dtype=np.float64).reshape(n, n)
    gx = np.clip(np.asarray(px) * n - 0.5, 0.0, n - 1.0)
    gy = np.clip(np.asarray(py) * n - 0.5, 0.0, n - 1.0)
    ix = np.minimum(np.floor(gx).astype(np.int64), max(n - 2, 0))
    iy = np.minimum(np.floor(gy).astype(np.int64), max(n - 2, 0))
    if n == 1:
        return np.full(np.shape(gx), S[0, 0])
    ax, ay = gx - ix, gy - iy
    v00, v10 = S[iy, ix], S[iy, ix + 1]
    v01, v11 = S[iy + 1, ix], S[iy + 1, ix + 1]
    return (1 - ay) * ((1 - ax) * v00 + ax * v10) + ay * ((1 - ax) * v01 + ax * v11)


def tau_march(sigma, n, x, y, S=64) -> np.ndarray:
    """(r / S) sum_i sigma~(x + (i + 1/2)/S (y - x)) for point arrays x, y [k, 2]."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    d = y - x
    t = (np.arange(S) + 0.5) / S
    px = x[:, 0:1] + t[None, :] * d[:, 0:1]
    py = x[:, 1:2] + t[None, :] * d[:, 1:2]
    r = np.hypot(d[:, 0], d[:, 1])
    return r / S * bilinear(sigma, n, px, py).sum(axis=1)


def kernel(sigma, n, x, y, S=64) -> np.ndarray:
    """K(x, y) = h^2 exp(-tau) / (2 pi r) for all pairs of point arrays: [len(x), len(y)]."""
    h = 1.0 / n
    X = np.repeat(x, len(y), axis=0)
    Y = np.tile(y, (len(x), 1))
    r = np.hypot(*(Y - X).T)
    return (h * h * np.exp(-tau_march(sigma, n, X, Y, S)) / (2 * np.pi * r)).reshape(len(x), len(y))


def _near_block(sigma, n, b, B, C, S):
    h = 1.0 / n
    cb = np.array([(B[0] * b + i % b + 0.5) * h for i in range(b * b)])
    rb = np.array([(B[1] * b + i // b + 0.5) * h for i in range(b * b)])
    cc = np.array([(C[0] * b + i % b + 0.5) * h for i in range(b * b)])
    rc = np.array([(C[1] * b + i // b + 0.5) * h for i in range(b * b)])
    xb = np.stack([cb, rb], 1)
    xc = np.stack([cc, rc], 1)
    X = np.repeat(xb, len(xc), axis=0)
    Y = np.tile(xc, (len(xb), 1))
    r = np.hypot(*(Y - X).T)
    same = r == 0
    r[same] = 1.0
    A = h * h * np.exp(-tau_march(sigma, n, X, Y, S)) / (2 * np.pi * r)
    A = A.reshape(len(xb), len(xc))
    if B == C:
        sig = np.asarray(sigma).reshape(n, n)
        for i in range(b * b):
            A[i, i] = selfcell(2, h, sig[B[1] * b + i // b, B[0] * b + i % b])
    return A


def interaction_list(level: int, B):
    """Boxes C at `level` in the far field of B whose parents are adjacent to (or
    equal to) B's parent."""
    nb = 2 ** level
    out = []
    px, py = B[0] // 2, B[1] // 2
    for cy in range(2 * py - 2, 2 * py + 4):
        for cx in range(2 * px - 2, 2 * px + 4):
            if 0 <= cx < nb and 0 <= cy < nb and (abs(cx - B[0]) > 1 or abs(cy - B[1]) > 1):
                out.append((cx, cy))
    return out


def apply(sigma_t, s, n: int, p: int, S: int = 64) -> np.ndarray:
    """y = A s by the FMM (y_j = sum_k A_jk s_k, A the M-iii matrix)."""
    L, b = leaf_levels(n)
    s = np.asarray(s, dtype=np.float64).reshape(n, n)
    y = np.zeros((n, n))
    nl = 2 ** L
    h = 1.0 / n
    # near field
    for by in range(nl):
        for bx in range(nl):
            acc = np.zeros(b * b)
            for cy in range(max(0, by - 1), min(nl, by + 2)):
                for cx in range(max(0, bx - 1), min(nl, bx + 2)):
                    A = _near_block(sigma_t, n, b, (bx, by), (cx, cy), S)
                    acc += A @ s[cy * b:(cy + 1) * b, cx * b:(cx + 1) * b].ravel()
            y[by * b:(by + 1) * b, bx * b:(bx + 1) * b] += acc.reshape(b, b)
    if L < 2:
        return y.ravel()
    # upward pass
    W = {}
    for by in range(nl):
        for bx in range(nl):
            pts = np.array([((bx * b + i % b + 0.5) * h, (by * b + i // b + 0.5) * h) for i in range(b * b)])
            M = interp_matrix(p, pts, (bx / nl, by / nl), 1.0 / nl)
            W[(L, bx, by)] = M @ s[by * b:(by + 1) * b, bx * b:(bx + 1) * b].ravel()
    for lev in range(L - 1, 1, -1):
        nb = 2 ** lev
        for by in range(nb):
            for bx in range(nb):
                acc = np.zeros(p * p)
                for q in range(4):
                    cx, cy = 2 * bx + q % 2, 2 * by + q // 2
                    nodes = box_nodes(p, (cx / (2 * nb), cy / (2 * nb)), 1.0 / (2 * nb))
                    acc += interp_matrix(p, nodes, (bx / nb, by / nb), 1.0 / nb) @ W[(lev + 1, cx, cy)]
                W[(lev, bx, by)] = acc
    # interactions
    Lc = {}
    for lev in range(2, L + 1):
        nb = 2 ** lev
        for by in range(nb):
            for bx in range(nb):
                tb = box_nodes(p, (bx / nb, by / nb), 1.0 / nb)
                acc = np.zeros(p * p)
                for (cx, cy) in interaction_list(lev, (bx, by)):
                    sc = box_nodes(p, (cx / nb, cy / nb), 1.0 / nb)
                    acc += kernel(sigma_t, n, tb, sc, S) @ W[(lev, cx, cy)]
                Lc[(lev, bx, by)] = acc
    # downward pass
    for lev in range(2, L):
        nb = 2 ** lev
        for by in range(nb):
            for bx in range(nb):
                for q in range(4):
                    cx, cy = 2 * bx + q % 2, 2 * by + q // 2
                    nodes = box_nodes(p, (cx / (2 * nb), cy / (2 * nb)), 1.0 / (2 * nb))
                    Lc[(lev + 1, cx, cy)] += interp_matrix(p, nodes, (bx / nb, by / nb), 1.0 / nb).T @ Lc[(lev, bx, by)]
    for by in range(nl):
        for bx in range(nl):
            pts = np.array([((bx * b + i % b + 0.5) * h, (by * b + i // b + 0.5) * h) for i in range(b * b)])
            M = interp_matrix(p, pts, (bx / nl, by / nl), 1.0 / nl)
            y[by * b:(by + 1) * b, bx * b:(bx + 1) * b] += (M.T @ Lc[(L, bx, by)]).reshape(b, b)
    return y.ravel()

