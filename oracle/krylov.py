"""Fine-grid solvers of the two-grid method, FP64, step by step in the paper's order.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  galerkin_project / minres_project   Section 2.2, "Galerkin projection over a set of
                                      approximate eigenvectors", and the MinRes variant
                                      stated right after it.
  bicgstab_cycle                      one cycle of BiCGStab (van der Vorst 1992, the
                                      textbook recurrence; the paper runs MATLAB's).
  cycle_tolerance                     Section 4.1, step 3b.
  bicgstab_proj                       BiCGStab(ncyc)-Proj(k), Section 4.1.
  gmres_cycle / gmres_proj            GMRES(m)-Proj(k), Section 2.2.
  idr_cycle / idr_proj                IDR(s) (van Gijzen and Sonneveld's biorthogonal IDR,
                                      the paper's other fine-grid solver) and
                                      IDR(ncyc)-Proj(k), Section 4.1.

Readings taken where the paper is silent:
  * ||r0|| in the cycle tolerance is ||b||, so "relative residual" is ||b - Ax|| / ||b||.
  * ||r|| in step 3b is the residual after step 3a's projection.
  * Each BiCGStab cycle starts with shadow vector r_hat = r, p = v = 0; it stops when
    ||r_it|| <= rticyc * ||r_cycle_start||, checked after the half step (s) and after the
    full step; it also stops after `restart_mvps` operator applications if that cap is
    set (fixed-length restarting, Example 2).
  * Breakdown (rho = 0, <r_hat, v> = 0, <t, t> = 0) ends the cycle early; the restart
    and the next projection are the remedy.  A cycle that ends before its first product
    ends the solve (nothing would change in the next one).
  * The true residual b - A x is recomputed at every restart.
  * Fixed-length mode (ncyc = 0): cycles of at most `restart_mvps` products, each with
    tolerance rtol ||b|| / ||r||, until convergence or `max_mvps`.
  * Past ncyc: the box loops icyc = 1..ncyc and says nothing of a solve whose last
    scheduled cycle ends above rtol (its recursive residual met rticyc while the true
    residual did not, or a breakdown or product cap ended it).  The solve then goes on
    with cycles whose tolerance is rtol ||b|| / ||r|| (the value step 3b gives at
    icyc = ncyc), until convergence or `max_mvps`.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

TINY = 1e-300


def dot(a, b):
    """<a, b> = a^H b (complex conjugate on the first argument)."""
    return np.vdot(a, b)


def nrm(a):
    return float(np.sqrt(np.vdot(a, a).real))


# ----------------------------------------------------------------------------- projections

@dataclass
class Deflation:
    """The k prolonged approximate eigenvectors and what each projection needs."""
    Y: np.ndarray             # n x k basis (columns)
    AY: np.ndarray            # n x k, A Y
    kind: str = "minres"      # "minres" or "galerkin"


def make_deflation(apply, Y: np.ndarray, kind: str = "minres") -> Deflation:
    """Form A Y (k operator applications, Section 3 Example 1 counts them)."""
    AY = np.stack([apply(Y[:, j]) for j in range(Y.shape[1])], axis=1)
    return Deflation(Y, AY, kind)


def galerkin_project(defl: Deflation, x, r):
    """Galerkin projection (Section 2.2 box): V orthonormal with span(V) = span(Y);
    H = V^T A V, c = V^T r0, solve H d = c, x += V d, r -= A V d."""
    V, Rf = np.linalg.qr(defl.Y)                 # Y = V Rf
    AV = np.linalg.solve(Rf.T, defl.AY.T).T      # A V = A Y Rf^{-1}
    H = V.conj().T @ AV
    c = V.conj().T @ r
    d = np.linalg.solve(H, c)
    return x + V @ d, r - AV @ d


def minres_project(defl: Deflation, x, r):
    """MinRes projection (Section 2.2): as Galerkin with H = (AV)^T AV, c = (AV)^T r0,
    i.e. d = argmin ||r0 - A Y d||, computed by Householder QR of A Y."""
    Q, R = np.linalg.qr(defl.AY)
    d = np.linalg.solve(R, Q.conj().T @ r)
    return x + defl.Y @ d, r - defl.AY @ d


def project(defl: Deflation, x, r):
    if defl is None or defl.Y.shape[1] == 0:
        return x, r
    if defl.kind == "galerkin":
        return galerkin_project(defl, x, r)
    return minres_project(defl, x, r)


# ----------------------------------------------------------------------------- BiCGStab

@dataclass
class CycleResult:
    x: np.ndarray
    r: np.ndarray
    mvps: int
    iters: int
    converged: bool
    breakdown: bool
    history: list = field(default_factory=list)


def bicgstab_cycle(apply, x, r, target, max_mvps=None):
    """One BiCGStab cycle on A e = r from e = 0, updating x and r in place of the
    caller's copies.  Stops when ||r|| <= target (checked at the half and full step),
    on breakdown, or after max_mvps operator applications."""
    x = x.copy()
    r = r.copy()
    r_hat = r.copy()
    p = np.zeros_like(r)
    v = np.zeros_like(r)
    rho_old = alpha = omega = 1.0
    mvps = 0
    iters = 0
    hist = []
    if nrm(r) <= target:
        return CycleResult(x, r, 0, 0, True, False, hist)
    while True:
        rho = dot(r_hat, r)
        if abs(rho) < TINY:
            return CycleResult(x, r, mvps, iters, False, True, hist)
        if iters == 0:
            p = r.copy()
        else:
            beta = (rho / rho_old) * (alpha / omega)
            p = r + beta * (p - omega * v)
        v = apply(p)
        mvps += 1
        sigma = dot(r_hat, v)
        if abs(sigma) < TINY:
            return CycleResult(x, r, mvps, iters, False, True, hist)
        alpha = rho / sigma
        s = r - alpha * v
        ns = nrm(s)
        hist.append(ns)
        if ns <= target or (max_mvps is not None and mvps >= max_mvps):
            x = x + alpha * p
            return CycleResult(x, s, mvps, iters + 1, ns <= target, False, hist)
        t = apply(s)
        mvps += 1
        tt = dot(t, t).real
        if tt < TINY:
            x = x + alpha * p
            return CycleResult(x, s, mvps, iters + 1, False, True, hist)
        omega = dot(t, s) / tt
        x = x + alpha * p + omega * s
        r = s - omega * t
        iters += 1
        nr = nrm(r)
        hist.append(nr)
        if nr <= target:
            return CycleResult(x, r, mvps, iters, True, False, hist)
        if abs(omega) < TINY:
            return CycleResult(x, r, mvps, iters, False, True, hist)
        if max_mvps is not None and mvps >= max_mvps:
            return CycleResult(x, r, mvps, iters, False, False, hist)
        rho_old = rho


def cycle_tolerance(rtol, nr0, nr, icyc, ncyc):
    """Section 4.1 step 3b: rticyc = min((rtol ||r0|| / ||r||)^(1/(ncyc-icyc+1)),
    (||r0|| / ||r||) rtol^(icyc/ncyc)), relative to the current ||r||."""
    a = (rtol * nr0 / nr) ** (1.0 / (ncyc - icyc + 1))
    b = (nr0 / nr) * rtol ** (icyc / ncyc)
    return min(a, b)


@dataclass
class SolveResult:
    x: np.ndarray
    converged: bool
    mvps: int
    cycles: int
    relres: float
    history: list = field(default_factory=list)   # (cycle, ||r||/||b|| after projection, rticyc, mvps)


def bicgstab_proj(apply, b, x0, defl: Deflation | None, rtol=1e-8, ncyc=20,
                  restart_mvps=None, max_mvps=100000):
    """BiCGStab(ncyc)-Proj(k), Section 4.1 step 3 (steps 1-2, the coarse phase and the
    move to the fine grid, produce x0 and defl).  ncyc = 0 selects fixed-length
    restarting every `restart_mvps` products."""
    nb = nrm(b)
    x = x0.copy()
    r = b - apply(x)
    mvps = 0
    hist = []
    icyc = 0
    while True:
        icyc += 1
        x, r = project(defl, x, r)                              # step a
        nr = nrm(r)
        if ncyc and icyc <= ncyc:
            rt = cycle_tolerance(rtol, nb, nr, icyc, ncyc)      # step b
        else:
            rt = rtol * nb / nr                                 # fixed-length mode, or past ncyc
        hist.append((icyc, nr / nb, rt, mvps))
        cap = restart_mvps if restart_mvps else None
        if cap is not None:
            cap = min(cap, max_mvps - mvps)
        res = bicgstab_cycle(apply, x, r, rt * nr, cap)        # step c
        x = res.x
        mvps += res.mvps
        r = b - apply(x)                                        # true residual at restart
        if nrm(r) <= rtol * nb:                                 # step d
            break
        if mvps >= max_mvps:
            break
        if res.mvps == 0:                                       # a cycle without progress
            break
    relres = nrm(b - apply(x)) / nb
    return SolveResult(x, relres <= rtol, mvps, icyc, relres, hist)


# ----------------------------------------------------------------------------- GMRES

def gmres_cycle(apply, x, r, m, target):
    """One GMRES(m) cycle from x (residual r): modified Gram-Schmidt Arnoldi, Givens
    rotations for the least-squares problem, exit as soon as the least-squares
    residual estimate is <= target (Example 1 notes this can be monitored in-cycle)."""
    n = r.shape[0]
    beta = nrm(r)
    if beta <= target:
        return CycleResult(x.copy(), r.copy(), 0, 0, True, False, [])
    V = np.zeros((n, m + 1), dtype=r.dtype)
    H = np.zeros((m + 1, m), dtype=r.dtype)
    V[:, 0] = r / beta
    cs = np.zeros(m, dtype=r.dtype)
    sn = np.zeros(m, dtype=r.dtype)
    g = np.zeros(m + 1, dtype=r.dtype)
    g[0] = beta
    j_done = 0
    hist = []
    for j in range(m):
        w = apply(V[:, j])
        for i in range(j + 1):
            H[i, j] = dot(V[:, i], w)
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = nrm(w)
        if H[j + 1, j] != 0:
            V[:, j + 1] = w / H[j + 1, j]
        for i in range(j):
            a, bb = H[i, j], H[i + 1, j]
            H[i, j] = np.conj(cs[i]) * a + np.conj(sn[i]) * bb
            H[i + 1, j] = -sn[i] * a + cs[i] * bb
        a, bb = H[j, j], H[j + 1, j]
        den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
        cs[j], sn[j] = a / den, bb / den
        H[j, j] = den
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = np.conj(cs[j]) * g[j]
        j_done = j + 1
        hist.append(abs(g[j + 1]))
        if abs(g[j + 1]) <= target or H[j, j] == 0:
            break
    k = j_done
    y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
    x = x + V[:, :k] @ y
    return CycleResult(x, None, k, k, abs(g[k]) <= target, False, hist)


def gmres_proj(apply, b, x0, defl: Deflation | None, m=20, rtol=1e-8, max_mvps=100000):
    """GMRES(m)-Proj(k), Section 2.2: alternate (A) a projection over the k vectors and
    (B) one GMRES(m) cycle, until ||b - Ax|| <= rtol ||b||."""
    nb = nrm(b)
    x = x0.copy()
    r = b - apply(x)
    mvps = 0
    cyc = 0
    hist = []
    while nrm(r) > rtol * nb and mvps < max_mvps:
        cyc += 1
        x, r = project(defl, x, r)                 # A)
        hist.append((cyc, nrm(r) / nb, None, mvps))
        res = gmres_cycle(apply, x, r, min(m, max_mvps - mvps), rtol * nb)   # B)
        x = res.x
        mvps += res.mvps
        r = b - apply(x)
    relres = nrm(b - apply(x)) / nb
    return SolveResult(x, relres <= rtol, mvps, cyc, relres, hist)


# ----------------------------------------------------------------------------- IDR(s)

def shadow_space(P_raw: np.ndarray) -> np.ndarray:
    """Orthonormal shadow space from random columns: the Q of the QR factorisation whose R
    has a positive diagonal (unique, so that any orthonormalisation with that convention
    gives the same P)."""
    Q, R = np.linalg.qr(P_raw)
    sg = np.sign(np.real(np.diag(R)))
    sg[sg == 0] = 1.0
    return Q * sg[None, :]


def idr_cycle(apply, x, r, P, target, max_mvps=None, kappa=0.7):
    """One cycle of IDR(s) from e = 0 on A e = r (updating copies of x and r), in the
    biorthogonal form of van Gijzen and Sonneveld (the IDR the paper runs, Section 4.1; s
    = P's column count, P orthonormal).  Stops when ||r|| <= target (checked after every
    residual update), on breakdown (M_kk = 0 or omega = 0), or after max_mvps products.

    Each round of s + 1 products:
      f = P^H r
      for k = 1..s:
        c = M[k:, k:]^{-1} f[k:]              (M lower triangular)
        v = r - G[:, k:] c
        U[:, k] = U[:, k:] c + omega v
        G[:, k] = A U[:, k]                   (one product)
        for i < k:  a = P_i^H G_k / M_ii;  G_k -= a G_i;  U_k -= a U_i
        M[k:, k] = P[:, k:]^H G_k
        beta = f_k / M_kk;  r -= beta G_k;  x += beta U_k
        f[k+1:] -= beta M[k+1:, k]
      t = A r                                  (one product)
      omega = <t, r> / <t, t>, enlarged to omega kappa / |rho| when the cosine
              rho = <t, r> / (||t|| ||r||) is below kappa in modulus
      x += omega r;  r -= omega t
    """
    x = x.copy()
    r = r.copy()
    n, s = P.shape
    G = np.zeros((n, s), dtype=r.dtype)
    U = np.zeros((n, s), dtype=r.dtype)
    M = np.eye(s, dtype=r.dtype)
    om = 1.0
    mvps = 0
    hist = []

    def cap_hit():
        return max_mvps is not None and mvps >= max_mvps

    if nrm(r) <= target:
        return CycleResult(x, r, 0, 0, True, False, hist)
    rounds = 0
    while True:
        f = P.conj().T @ r
        for k in range(s):
            c = np.linalg.solve(np.tril(M[k:, k:]), f[k:])
            v = r - G[:, k:] @ c
            U[:, k] = U[:, k:] @ c + om * v
            G[:, k] = apply(U[:, k])
            mvps += 1
            for i in range(k):
                a = dot(P[:, i], G[:, k]) / M[i, i]
                G[:, k] = G[:, k] - a * G[:, i]
                U[:, k] = U[:, k] - a * U[:, i]
            M[k:, k] = P[:, k:].conj().T @ G[:, k]
            if abs(M[k, k]) < TINY:
                return CycleResult(x, r, mvps, rounds, False, True, hist)
            beta = f[k] / M[k, k]
            r = r - beta * G[:, k]
            x = x + beta * U[:, k]
            nr = nrm(r)
            hist.append(nr)
            if nr <= target:
                return CycleResult(x, r, mvps, rounds, True, False, hist)
            if cap_hit():
                return CycleResult(x, r, mvps, rounds, False, False, hist)
            if k + 1 < s:
                f[k + 1:] = f[k + 1:] - beta * M[k + 1:, k]
        t = apply(r)
        mvps += 1
        tt = dot(t, t).real
        if tt < TINY:
            return CycleResult(x, r, mvps, rounds, False, True, hist)
        tr = dot(t, r)
        om = tr / tt
        rho = abs(tr) / np.sqrt(tt * dot(r, r).real)
        if rho < kappa:
            om = om * kappa / rho
        if abs(om) < TINY:
            return CycleResult(x, r, mvps, rounds, False, True, hist)
        x = x + om * r
        r = r - om * t
        rounds += 1
        nr = nrm(r)
        hist.append(nr)
        if nr <= target:
            return CycleResult(x, r, mvps, rounds, True, False, hist)
        if cap_hit():
            return CycleResult(x, r, mvps, rounds, False, False, hist)


def idr_proj(apply, b, x0, defl: Deflation | None, P, rtol=1e-8, ncyc=20, restart_mvps=None,
             max_mvps=100000, kappa=0.7):
    """IDR(ncyc)-Proj(k), Section 4.1 step 3 with IDR(s) in place of BiCGStab: the same
    cycle schedule (projection, rticyc, a cycle of IDR(s) to rticyc, true residual), with
    the same readings as bicgstab_proj (||r0|| = ||b||, cycles past ncyc aim at rtol, one
    shadow space P for every cycle)."""
    nb = nrm(b)
    x = x0.copy()
    r = b - apply(x)
    mvps = 0
    hist = []
    icyc = 0
    while True:
        icyc += 1
        x, r = project(defl, x, r)                              # step a
        nr = nrm(r)
        if ncyc and icyc <= ncyc:
            rt = cycle_tolerance(rtol, nb, nr, icyc, ncyc)      # step b
        else:
            rt = rtol * nb / nr
        hist.append((icyc, nr / nb, rt, mvps))
        cap = max_mvps - mvps
        if restart_mvps:
            cap = min(cap, restart_mvps)
        res = idr_cycle(apply, x, r, P, rt * nr, cap, kappa)    # step c
        x = res.x
        mvps += res.mvps
        r = b - apply(x)
        if nrm(r) <= rtol * nb:                                 # step d
            break
        if mvps >= max_mvps or res.mvps == 0:
            break
    relres = nrm(b - apply(x)) / nb
    return SolveResult(x, relres <= rtol, mvps, icyc, relres, hist)
