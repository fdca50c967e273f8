"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle and the benchmark.

This module draws random numbers and lays them out; it holds none of the solver's
arithmetic (no operator, no interpolation, no Krylov step), so both sides of every
parity check can take their inputs from here without sharing any of the method.

Workloads follow the paper's test problems: PDE discretisations on the unit square
or cube with random-normal right-hand sides (Example 3, Example 4, Example 6), and a
lattice operator with random U(1) link phases standing in for the Schwinger-model
gauge fields of Example 8.

Layouts:
  * 2D grid vectors: length N*N, index (j-1)*N + (i-1), x (i) fastest.
  * 3D grid vectors: length N^3, index (i-1) + N*((j-1) + N*(k-1)).
  * kappa for the variable-coefficient operator: the (N+2)^2 node grid including
    the Dirichlet boundary nodes, index j*(N+2) + i, i, j in 0..N+1.
  * 4D lattice: V = L^4 sites, index x0 + L*(x1 + L*(x2 + L*x3)); links U[mu][site],
    complex128, mu = 0..3.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rhs", "u1_links", "kappa_grf", "batch_instances", "kappa_fd_nodes",
    "random_dense", "random_hessenberg", "example1_rhs",
]


def _rng(seed: int, stream: int) -> np.random.Generator:
    # one independent stream per (seed, purpose) so that drawing one input never
    # shifts another
    return np.random.default_rng([int(seed), int(stream)])


def rhs(n: int, seed: int = 0, nrhs: int = 1) -> np.ndarray:
    """Right-hand side(s) b ~ N(0, 1), float64.  Shape (n,) or (nrhs, n)."""
    g = _rng(seed, 1)
    if nrhs == 1:
        return g.standard_normal(n)
    return g.standard_normal((nrhs, n))


def u1_links(L: int, seed: int = 0) -> np.ndarray:
    """U(1) gauge links U_mu(x) = exp(i theta), theta ~ U(-pi, pi); shape (4, L^4) complex128."""
    g = _rng(seed, 2)
    theta = g.uniform(-np.pi, np.pi, size=(4, L ** 4))
    return np.exp(1j * theta)


def kappa_grf(N: int, seed: int = 0, length: float = 0.1, sigma: float = 1.0) -> np.ndarray:
    """kappa = exp(GRF) on the (N+2)^2 node grid of the unit square (h = 1/(N+1)).

    The field has squared-exponential covariance sigma^2 exp(-r^2 / (2 length^2)).  It is
    drawn by circulant embedding: the covariance is laid on a periodic M x M grid with
    M >= 2 (N+2), its FFT gives the spectrum (negative parts clipped), white complex
    noise shaped by the square root of the spectrum is transformed back, and the
    (N+2) x (N+2) corner is kept.  Returned flat, index j*(N+2) + i, float64.
    """
    g = _rng(seed, 3)
    n1 = N + 2
    M = 1
    while M < 2 * n1:
        M *= 2
    h = 1.0 / (N + 1)
    d = np.minimum(np.arange(M), M - np.arange(M)) * h
    r2 = d[:, None] ** 2 + d[None, :] ** 2
    cov = sigma ** 2 * np.exp(-r2 / (2.0 * length ** 2))
    lam = np.fft.fft2(cov).real
    lam = np.maximum(lam, 0.0)
    xi = g.standard_normal((M, M)) + 1j * g.standard_normal((M, M))
    field = np.fft.ifft2(np.sqrt(lam) * xi) * M  # unit-variance normalisation of ifft2
    z = field.real[:n1, :n1]
    return np.exp(z).reshape(-1).copy()


def batch_instances(count: int = 128, seed: int = 0, nmin: int = 255, nmax: int = 1023):
    """Sizes and convection speeds of independent 2D problems: N odd in [nmin, nmax],
    beta ~ U(0.5, 4).  Odd N keeps the coarse grid (N-1)/2 nested."""
    g = _rng(seed, 4)
    odd = np.arange(nmin | 1, nmax + 1, 2)
    Ns = g.choice(odd, size=count)
    betas = g.uniform(0.5, 4.0, size=count)
    return [int(v) for v in Ns], [float(v) for v in betas]


def kappa_fd_nodes(N: int, count: int = 64, seed: int = 0) -> np.ndarray:
    """`count` distinct interior kappa nodes (flat (N+2)^2 indices) for finite-difference checks."""
    g = _rng(seed, 5)
    flat = g.choice(N * N, size=count, replace=False)
    i = flat % N + 1
    j = flat // N + 1
    return (j * (N + 2) + i).astype(np.int64)


def random_dense(shape, seed: int = 0) -> np.ndarray:
    """Dense N(0, 1) float64 array (test matrices, bases, vectors)."""
    return _rng(seed, 6).standard_normal(shape)


def random_hessenberg(m: int, seed: int = 0, rows: int | None = None) -> np.ndarray:
    """(rows x m) upper-Hessenberg N(0, 1) matrix (rows defaults to m + 1)."""
    rows = m + 1 if rows is None else rows
    a = _rng(seed, 7).standard_normal((rows, m))
    for c in range(m):
        a[c + 2:, c] = 0.0
    return a


def example1_rhs(N: int) -> np.ndarray:
    """Right-hand side of the paper's Example 1 as printed, f = c sin(x) cos(x) exp(x y) on the
    interior nodes x = i h, y = j h (h = 1/(N+1)), x fastest, c making ||f|| = 1."""
    h = 1.0 / (N + 1)
    t = np.arange(1, N + 1) * h
    Y, X = np.meshgrid(t, t, indexing="ij")
    f = (np.sin(X) * np.cos(X) * np.exp(X * Y)).reshape(-1)
    return f / np.linalg.norm(f)
