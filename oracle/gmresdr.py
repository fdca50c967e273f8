"""GMRES-DR(m,k) (GMRES with deflated restarting), FP64, in the paper's notation.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 2.1: each cycle after the first works in span{y_1..y_k, r0, A r0, ...,
A^{m-k-1} r0}, with y_i the harmonic Ritz vectors of the previous cycle and r0 the
residual at the start of the cycle.  The cycle structure written out here is Morgan's
published GMRES-DR (the method the paper cites):

  cycle 1: GMRES(m) from x0 -> V_{m+1}, Hbar_m; d = argmin ||c - Hbar_m d||, c = beta e1.
  restart: harmonic Ritz pairs (theta, g) of Hbar_m are the eigenpairs of
           H_m + |h_{m+1,m}|^2 f e_m^T with H_m^H f = e_m; keep the k of smallest |theta|;
           P_k = orthonormal basis of their (real) span; P_{k+1} = [P_k; 0] extended by the
           least-squares residual c - Hbar_m d (in the direction z, see
           residual_direction); V_{k+1} <- V_{m+1} P_{k+1};
           Hbar_k <- P_{k+1}^H Hbar_m P_k; c <- P_{k+1}^H (c - Hbar_m d); then Arnoldi
           extends V to m + 1 columns and the least-squares problem is solved again.

Readings taken:
  * Order of the harmonic Ritz values: by |theta|, then Re theta, then Im theta >= 0 first.
    If the k-th value splits a complex-conjugate pair, k + 1 are kept for that cycle.
  * Real problems keep a real basis: Re g and Im g of each kept complex pair.
  * The eigen-residual of a pair is ||A y - theta y|| = ||Hbar_m g - theta [g; 0]|| with
    ||g|| = 1 (computed only at the end of cycles, Example 1); a pair has converged when
    that residual is <= rtolev |theta| (relative: the paper's scaling of A is not stated).
  * Stop when the linear residual is <= rtol ||b|| and the nev smallest pairs have
    converged, or after max_cycles.
  * The (k+1)-th restart direction is z = [-|h_{m+1,m}|^2 f; h_{m+1,m}], parallel to the
    least-squares residual in exact arithmetic (both span range(Hbar_m)^perp) but
    computed from Hbar alone, so the restart relation A V_k = V_{k+1} Hbar_k survives
    after the linear system has converged.
  * The basis handed to the fine grid is the orthonormal V_m P_k of the final cycle: the
    projection depends only on span(Y), and this span is that of the harmonic Ritz
    vectors, without complex arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def harmonic_ritz(Hbar: np.ndarray):
    """All harmonic Ritz pairs of an (m+1) x m Hessenberg Hbar (library eig as one step)."""
    m = Hbar.shape[1]
    Hm = Hbar[:m, :m]
    em = np.zeros(m, dtype=Hbar.dtype)
    em[-1] = 1.0
    f = np.linalg.solve(Hm.conj().T, em)
    M = Hm.astype(np.complex128 if np.iscomplexobj(Hbar) else np.float64).copy()
    M[:, -1] += abs(Hbar[m, m - 1]) ** 2 * f
    theta, G = np.linalg.eig(M)
    return theta, G


def order_ritz(theta: np.ndarray) -> np.ndarray:
    """Indices sorted by |theta|, then Re theta, then Im theta >= 0 first."""
    keys = [(abs(t), t.real, 0 if t.imag >= 0 else 1) for t in theta]
    return np.array(sorted(range(len(theta)), key=lambda i: keys[i]), dtype=np.int64)


def select_k(theta: np.ndarray, k: int, real_problem: bool):
    """The kept indices: k smallest in the order above, k+1 if a conjugate pair would split."""
    order = order_ritz(theta)
    kk = k
    if real_problem and kk < len(order):
        t = theta[order[kk - 1]]
        if abs(t.imag) > 0 and t.imag > 0:
            kk += 1
    return order[:kk]


def real_span_basis(G: np.ndarray, theta: np.ndarray, idx: np.ndarray, real_problem: bool):
    """m x kk matrix whose columns span the kept eigenvectors (Re/Im of complex pairs)."""
    if not real_problem:
        return G[:, idx]
    cols = []
    for i in idx:
        if theta[i].imag == 0:
            cols.append(G[:, i].real)
        elif theta[i].imag > 0:
            cols.append(G[:, i].real)
            cols.append(G[:, i].imag)
        # Im < 0: the partner (Im > 0) supplies both columns
    return np.stack(cols, axis=1)


def residual_direction(Hbar: np.ndarray) -> np.ndarray:
    """z = [-|h_{m+1,m}|^2 f; h_{m+1,m}] with H_m^H f = e_m.

    Hbar^H z = 0, so z spans the one-dimensional complement of range(Hbar_m): the
    least-squares residual c - Hbar_m d and every harmonic Ritz residual
    Hbar_m g - theta [g; 0] = (e_m^T g) z are parallel to it.  Using z (rather than the
    least-squares residual itself) as the (k+1)-th restart direction gives the same
    span in exact arithmetic and stays well defined once the linear residual has
    reached rounding level and its direction is noise."""
    m = Hbar.shape[1]
    em = np.zeros(m, dtype=Hbar.dtype)
    em[-1] = 1.0
    f = np.linalg.solve(Hbar[:m, :m].conj().T, em)
    hm = Hbar[m, m - 1]
    return np.concatenate([-abs(hm) ** 2 * f, [hm]])


def eigen_residuals(Hbar, theta, G, idx):
    """||Hbar g - theta [g; 0]|| / ||g|| for the pairs in idx."""
    m = Hbar.shape[1]
    out = []
    for i in idx:
        g = G[:, i] / np.linalg.norm(G[:, i])
        gz = np.zeros(m + 1, dtype=np.complex128)
        gz[:m] = g
        out.append(np.linalg.norm(Hbar @ g - theta[i] * gz))
    return np.array(out)


def arnoldi_extend(apply, V, H, j0, m):
    """Extend the Arnoldi relation A V_j = V_{j+1} Hbar_j from column j0 to m (classical
    Gram-Schmidt applied twice, written as two projections)."""
    for j in range(j0, m):
        w = apply(V[:, j])
        h = V[:, :j + 1].conj().T @ w
        w = w - V[:, :j + 1] @ h
        h2 = V[:, :j + 1].conj().T @ w
        w = w - V[:, :j + 1] @ h2
        H[:j + 1, j] = h + h2
        H[j + 1, j] = np.linalg.norm(w)
        V[:, j + 1] = w / H[j + 1, j]
    return V, H


@dataclass
class GmresDrResult:
    x: np.ndarray
    Yc: np.ndarray               # n_c x kk orthonormal basis of the final harmonic Ritz span
    theta: np.ndarray            # kept harmonic Ritz values (final cycle), in order
    eig_res: np.ndarray          # their residual norms
    cycles: int
    mvps: int
    relres: float
    converged: bool
    history: list = field(default_factory=list)   # per cycle: (relres, #eig converged)


def gmresdr(apply, b, m, k, nev=None, rtolev=1e-6, rtol=1e-8, max_cycles=300, x0=None,
            dtype=np.float64):
    """GMRES-DR(m,k) on A x = b (Section 2.1).  Returns the solution and the basis."""
    nev = k if nev is None else nev
    real_problem = not np.issubdtype(dtype, np.complexfloating)
    n = b.shape[0]
    x = np.zeros(n, dtype=dtype) if x0 is None else x0.astype(dtype).copy()
    nb = np.linalg.norm(b)
    r = b - apply(x) if x0 is not None else b.astype(dtype).copy()
    mvps = 1 if x0 is not None else 0
    V = np.zeros((n, m + 1), dtype=dtype)
    H = np.zeros((m + 1, m), dtype=dtype)
    beta = np.linalg.norm(r)
    V[:, 0] = r / beta
    c = np.zeros(m + 1, dtype=dtype)
    c[0] = beta
    j0 = 0
    hist = []
    cycles = 0
    while True:
        cycles += 1
        V, H = arnoldi_extend(apply, V, H, j0, m)
        mvps += m - j0
        d = np.linalg.lstsq(H, c, rcond=None)[0]
        x = x + V[:, :m] @ d
        res = c - H @ d
        rn = np.linalg.norm(res)
        theta, G = harmonic_ritz(H)
        idx = select_k(theta, k, real_problem)
        eres = eigen_residuals(H, theta, G, idx)
        nconv = int(np.sum(eres[:nev] <= rtolev * np.abs(theta[idx[:nev]])))
        hist.append((rn / nb, nconv))
        done = (rn <= rtol * nb and nconv >= nev) or cycles >= max_cycles
        Pk = np.linalg.qr(real_span_basis(G, theta, idx, real_problem))[0].astype(dtype)
        kk = Pk.shape[1]
        if done:
            Yc = V[:, :m] @ Pk
            return GmresDrResult(x, Yc, theta[idx], eres, cycles, mvps, rn / nb,
                                 rn <= rtol * nb and nconv >= nev, hist)
        # restart: P_{k+1} = [[P_k; 0], z] orthonormalised, z spanning range(Hbar_m)^perp
        Pk1 = np.zeros((m + 1, kk + 1), dtype=dtype)
        Pk1[:m, :kk] = Pk
        Pk1[:, kk] = residual_direction(H)
        Pk1 = np.linalg.qr(Pk1)[0]
        Vn = V @ Pk1
        Hn = Pk1.conj().T @ H @ Pk1[:m, :kk]
        cn = Pk1.conj().T @ res
        # re-orthogonalise v_{k+1} against V_k
        w = Vn[:, kk]
        w = w - Vn[:, :kk] @ (Vn[:, :kk].conj().T @ w)
        Vn[:, kk] = w / np.linalg.norm(w)
        V = np.zeros((n, m + 1), dtype=dtype)
        H = np.zeros((m + 1, m), dtype=dtype)
        V[:, :kk + 1] = Vn
        H[:kk + 1, :kk] = Hn
        c = np.zeros(m + 1, dtype=dtype)
        c[:kk + 1] = cn
        j0 = kk


# ----------------------------------------------------------------------------- Arnoldi-E

def rayleigh_ritz(S, AS, k, real_problem):
    """Ritz pairs of span(S) (S orthonormal, AS = A S): eigenpairs of H = S^H A S, ordered
    as the harmonic Ritz values above, k kept (k + 1 if a pair would split).  Returns
    (theta of all pairs in order, kept indices into that order, eigenvectors G of H,
    the residual norms ||A S g - theta S g|| of the kept pairs, ||g|| = 1)."""
    H = S.conj().T @ AS
    theta, G = np.linalg.eig(H)
    idx = select_k(theta, k, real_problem)
    eres = []
    for i in idx:
        g = G[:, i] / np.linalg.norm(G[:, i])
        eres.append(np.linalg.norm(AS @ g - theta[i] * (S @ g)))
    return theta, idx, G, np.array(eres)


def start_vector(S, G, i, real_problem):
    """The Ritz vector S g_i with the largest entry of g_i made real and positive (the
    smallest index on ties); real problems take its real part; unit norm."""
    g = G[:, i]
    j = int(np.argmax(np.abs(g)))
    g = g * (np.conj(g[j]) / abs(g[j]))
    if real_problem:
        g = g.real
    u = S @ g
    return u / np.linalg.norm(u)


def arnoldi_e(apply, Y, m, cycles, nstart, nev=0, rtolev=0.0, dtype=np.float64):
    """Arnoldi-E(m, k) improvement of k approximate eigenvectors (the paper's phase 2,
    Section 3 box step 2 and Section 4.1 box step 2, Example 7: "Arnoldi-E(150,100) ...
    with the 10 smallest approximate eigenvectors used as starting vectors").

    Readings taken (the paper defers to its Arnoldi-E reference):
      * a Rayleigh-Ritz step on span(Y) first orders the given vectors as Ritz vectors;
      * cycle c works in S = span{u, A u, ..., A^(m-k) u} + span(Y), u the Ritz vector
        number (c mod nstart) of the previous step (smallest first), of dimension m
        (u lies in span(Y), so one appended direction is dependent and dropped);
      * Rayleigh-Ritz on S (standard Ritz values, ordered and selected like the harmonic
        ones of GMRES-DR), Y <- orthonormal real basis of the kept span;
      * stop after `cycles` cycles, or earlier once the nev smallest pairs have residual
        <= rtolev |theta| (rtolev > 0).
    Returns (Y, theta of the kept pairs, their residual norms, cycles run, products)."""
    real_problem = not np.issubdtype(dtype, np.complexfloating)
    n, k = Y.shape
    p = m - k
    S = np.linalg.qr(Y)[0]
    AS = np.stack([apply(S[:, j]) for j in range(k)], axis=1)
    mvps = k
    theta, idx, G, eres = rayleigh_ritz(S, AS, k, real_problem)
    basis = np.linalg.qr(real_span_basis(G, theta, idx, real_problem))[0]
    Y = S @ basis
    u = start_vector(S, G, idx[0 % nstart], real_problem)
    done = 0
    for c in range(cycles):
        # Krylov part from u (Arnoldi, classical Gram-Schmidt twice), then span(Y)
        V = np.zeros((n, p + 1), dtype=dtype)
        Hk = np.zeros((p + 1, p), dtype=dtype)
        V[:, 0] = u
        V, Hk = arnoldi_extend(apply, V, Hk, 0, p)
        mvps += p
        cols = [V[:, j] for j in range(p + 1)]
        for j in range(Y.shape[1]):
            w = Y[:, j].copy()
            w0 = np.linalg.norm(w)
            Q = np.stack(cols, axis=1)
            for _ in range(2):
                w = w - Q @ (Q.conj().T @ w)
            if np.linalg.norm(w) > 1e-10 * w0:
                cols.append(w / np.linalg.norm(w))
        S = np.stack(cols, axis=1)
        AS = np.stack([apply(S[:, j]) for j in range(S.shape[1])], axis=1)
        mvps += S.shape[1]
        theta, idx, G, eres = rayleigh_ritz(S, AS, k, real_problem)
        basis = np.linalg.qr(real_span_basis(G, theta, idx, real_problem))[0]
        Y = S @ basis
        done = c + 1
        nconv = int(np.sum(eres[:nev] <= rtolev * np.abs(theta[idx[:nev]]))) if rtolev > 0 else 0
        if rtolev > 0 and nconv >= nev:
            break
        u = start_vector(S, G, idx[(c + 1) % nstart], real_problem)
    return Y, theta[idx], eres, done, mvps
