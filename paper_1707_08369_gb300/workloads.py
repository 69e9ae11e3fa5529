"""Seeded synthetic inputs for the rank-one SVD update.

This module only draws random numbers and builds test matrices; it holds none
of the update's arithmetic.  The paper measures on random matrices only
(Sec. 7: square, entries uniform in [1, 9]; Sec. 7.1: 25x25, entries uniform
in [0, 1]); the larger workloads below stand in for those at scale.

Every generator takes an explicit seed and returns float64 numpy arrays
(column-major where a matrix is returned), so the CPU oracle and the CUDA
library can be fed byte-identical inputs.

Workloads (seed = 170708369 + index):
  small_gaussian   64x64 N(0,1) matrix A and N(0,1) a, b (its SVD is taken by
                   the caller, e.g. with the oracle's Jacobi SVD).
  graded_rect      2048x4096, A = U diag(sigma) V^T, Haar U, V,
                   sigma_i = 10^(-6 i / 2048), 5% of sigma duplicated as
                   near-equal pairs (gap 1e-13), N(0,1) a, b.
  loguniform_sq    n x n (n = 8192 at full size), Haar U, V, sigma log-uniform
                   in [1e-4, 1] (sorted descending), N(0,1) a, b.
  uneven_batch     independent square problems, n log-uniform in [32, 1024].
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 170708369


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


def haar(n: int, g: np.random.Generator, device=None) -> np.ndarray:
    """Haar-distributed orthogonal n x n matrix: QR of a Gaussian matrix with the
    signs of R's diagonal moved into Q (Mezzadri 2007).  With ``device`` set (a
    torch CUDA device) the QR runs there; the Gaussian is always drawn by numpy."""
    G = g.standard_normal((n, n))
    if device is None:
        return haar_from_gaussian(G)
    import torch
    Gt = torch.from_numpy(G).to(device)
    try:
        Q, R = torch.linalg.qr(Gt)
    except RuntimeError:  # no device linear-algebra library in this torch build
        del Gt
        return haar_from_gaussian(G)
    s = torch.sign(torch.diagonal(R))
    s[s == 0] = 1.0
    Q = Q * s
    out = Q.cpu().numpy()
    del Gt, Q, R
    return np.asfortranarray(out)


def haar_from_gaussian(G: np.ndarray) -> np.ndarray:
    Q, R = np.linalg.qr(G)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return np.asfortranarray(Q * s)


def small_gaussian(m: int = 64, n: int = 64, seed: int = BASE_SEED + 0):
    """A (m x n), a (m), b (n), all N(0,1)."""
    g = rng(seed)
    A = np.asfortranarray(g.standard_normal((m, n)))
    a = g.standard_normal(m)
    b = g.standard_normal(n)
    return A, a, b


def uniform_square(n: int, lo: float, hi: float, seed: int):
    """The paper's experiment shape (Sec. 7): square A and vectors a, b with
    entries uniform in [lo, hi]."""
    g = rng(seed)
    A = np.asfortranarray(g.uniform(lo, hi, (n, n)))
    a = g.uniform(lo, hi, n)
    b = g.uniform(lo, hi, n)
    return A, a, b


def graded_sigma(m: int, g: np.random.Generator, decades: float = 6.0,
                 pair_frac: float = 0.05, gap: float = 1e-13) -> np.ndarray:
    """sigma_i = 10^(-decades i/m), then pair_frac*m seeded indices get a
    near-equal partner sigma_{i+1} = sigma_i - gap; returned descending."""
    s = 10.0 ** (-decades * np.arange(m) / m)
    npairs = int(round(pair_frac * m))
    if npairs:
        cand = np.arange(0, m - 1, 2)
        idx = g.choice(cand, size=min(npairs, cand.size), replace=False)
        for i in idx:
            s[i + 1] = s[i] - gap
    return np.sort(s)[::-1].copy()


def loguniform_sigma(m: int, g: np.random.Generator, lo: float = 1e-4, hi: float = 1.0) -> np.ndarray:
    u = g.uniform(0.0, 1.0, m)
    s = lo * (hi / lo) ** u
    return np.sort(s)[::-1].copy()


def svd_problem(m: int, n: int, sigma: np.ndarray, seed: int, device=None):
    """(U, S, V, a, b) with Haar U (m x m), V (n x n), given sigma, N(0,1) a, b."""
    g = rng(seed)
    U = haar(m, g, device)
    V = haar(n, g, device)
    a = g.standard_normal(m)
    b = g.standard_normal(n)
    return U, np.ascontiguousarray(sigma, dtype=np.float64), V, a, b


def graded_rect(m: int = 2048, n: int = 4096, seed: int = BASE_SEED + 1, device=None):
    g = rng(seed + 1000)
    sigma = graded_sigma(m, g)
    return svd_problem(m, n, sigma, seed, device)


def loguniform_sq(n: int = 8192, seed: int = BASE_SEED + 2, device=None):
    g = rng(seed + 1000)
    sigma = loguniform_sigma(n, g)
    return svd_problem(n, n, sigma, seed, device)


def uneven_sizes(count: int = 512, lo: int = 32, hi: int = 1024, seed: int = BASE_SEED + 3):
    g = rng(seed)
    u = g.uniform(0.0, 1.0, count)
    return np.rint(lo * (hi / lo) ** u).astype(np.int64)


def random_vectors(m: int, n: int, seed: int):
    g = rng(seed)
    return g.standard_normal(m), g.standard_normal(n)
