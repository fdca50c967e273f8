"""Discrete operators of the test problems, FP64, written out from their definitions.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper solves A x = b from finite-difference discretisations of PDEs on the unit
square with zero Dirichlet boundaries (Section 1; Example 1, Section 3; Example 4,
Section 5.1) and a lattice operator (Example 8, Section 5.4).  The operators here:

  cd2d   -u_xx - u_yy + beta u_x + c u, 5-point centred differences, h = 1/(N+1)
  cd3d   -Lap u + beta . grad u + c u, 7-point centred differences
  exp2d  -exp(gamma x y)(u_xx + u_yy) + beta_x u_x + beta_y u_y + c u at x = i h, y = j h
         (Example 1: gamma = 5, beta = (40, 40)); beta = (beta_x, beta_y, gamma)
  vark2d -div(kappa grad u) + beta u_x, kappa on the nodes, arithmetic face means

The reaction coefficient c (field `mass` on the grid kinds, 0 by default) gives the
Helmholtz operator of Example 4, -u_xx - u_yy - 100^2 u, as cd2d with beta = 0, c = -1e4.
  u1_4d  (m + 8) psi(x) - sum_mu [U_mu(x) psi(x+mu) + conj(U_mu(x-mu)) psi(x-mu)],
         periodic L^4 lattice, complex128

Scaling reading: true 1/h^2 scaling (the paper does not state its scaling; relative
residuals and Krylov iterates do not depend on it).

Each operator is available matrix-free (``apply``) and as a scipy sparse matrix
(``assemble``), built independently from the same stencil definition so that one can
check the other.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

CD2D, CD3D, U1_4D, VARK2D, EXP2D = 0, 1, 2, 3, 4


@dataclass
class Operator:
    kind: int
    N: int                       # interior points per axis (grids) or L (lattice)
    beta: tuple = (0.0,)         # convection speeds (cd2d/vark2d: (bx,), cd3d: (bx, by, bz),
                                 # exp2d: (bx, by, gamma))
    kappa: np.ndarray | None = None   # vark2d: (N+2)^2 node values
    links: np.ndarray | None = None   # u1_4d: (4, L^4) complex links
    mass: float = 0.0                 # u1_4d: the mass m; cd2d/cd3d/exp2d: reaction coefficient c
    transpose: bool = False           # exp2d: apply A^T (the other kinds form A^T by their parameters)
    _sparse: object = field(default=None, repr=False)

    @property
    def n(self) -> int:
        if self.kind in (CD2D, VARK2D, EXP2D):
            return self.N * self.N
        if self.kind == CD3D:
            return self.N ** 3
        return self.N ** 4

    @property
    def dtype(self):
        return np.complex128 if self.kind == U1_4D else np.float64

    def transposed(self) -> "Operator":
        """A^T for the real operators.  For centred convection with a symmetric
        diffusion part, A^T is the same operator with beta negated; this is checked
        against the sparse transpose by the tests, not assumed."""
        if self.kind == U1_4D:
            raise ValueError("the lattice operator is Hermitian; use the conjugate transpose")
        if self.kind == EXP2D:
            return Operator(EXP2D, self.N, self.beta, None, None, self.mass, transpose=not self.transpose)
        return Operator(self.kind, self.N, tuple(-b for b in self.beta), self.kappa, None, self.mass)

    def apply(self, u: np.ndarray) -> np.ndarray:
        return {CD2D: _apply_cd2d, CD3D: _apply_cd3d, VARK2D: _apply_vark2d,
                U1_4D: _apply_u1, EXP2D: _apply_exp2d}[self.kind](self, u)

    def sparse(self):
        if self._sparse is None:
            self._sparse = {CD2D: _assemble_cd2d, CD3D: _assemble_cd3d,
                            VARK2D: _assemble_vark2d, U1_4D: _assemble_u1,
                            EXP2D: _assemble_exp2d}[self.kind](self)
        return self._sparse


# ----------------------------------------------------------------------------- 2D / 3D

def _apply_cd2d(op: Operator, u):
    N = op.N
    h = 1.0 / (N + 1)
    bx = op.beta[0]
    U = np.zeros((N + 2, N + 2))
    U[1:-1, 1:-1] = u.reshape(N, N)          # [j, i], x fastest
    c = U[1:-1, 1:-1]
    xm, xp = U[1:-1, :-2], U[1:-1, 2:]
    ym, yp = U[:-2, 1:-1], U[2:, 1:-1]
    Au = (4.0 * c - xm - xp - ym - yp) / h**2 + bx * (xp - xm) / (2.0 * h) + op.mass * c
    return Au.reshape(-1)


def _exp2d_a(N, gamma):
    """The diffusion coefficient exp(gamma x y) at the interior nodes, [j, i], x = i h, y = j h."""
    h = 1.0 / (N + 1)
    t = np.arange(1, N + 1) * h
    return np.exp(gamma * t[:, None] * t[None, :])     # symmetric in (x, y)


def _apply_exp2d(op: Operator, u):
    """A u = a (-Lap_h u) + bx D_x u + by D_y u + c u with a = exp(gamma x y); the transpose
    is A^T u = -Lap_h (a u) - bx D_x u - by D_y u + c u (-Lap_h is symmetric, the centred
    differences antisymmetric)."""
    N = op.N
    h = 1.0 / (N + 1)
    bx, by, gamma = op.beta
    a = _exp2d_a(N, gamma)
    uu = u.reshape(N, N)
    U = np.zeros((N + 2, N + 2))
    U[1:-1, 1:-1] = a * uu if op.transpose else uu
    lap = (4.0 * U[1:-1, 1:-1] - U[1:-1, :-2] - U[1:-1, 2:] - U[:-2, 1:-1] - U[2:, 1:-1]) / h**2
    V = np.zeros((N + 2, N + 2))
    V[1:-1, 1:-1] = uu
    conv = (bx * (V[1:-1, 2:] - V[1:-1, :-2]) + by * (V[2:, 1:-1] - V[:-2, 1:-1])) / (2.0 * h)
    if op.transpose:
        Au = lap - conv
    else:
        Au = a * lap + conv
    return (Au + op.mass * uu).reshape(-1)


def _apply_cd3d(op: Operator, u):
    N = op.N
    h = 1.0 / (N + 1)
    bx, by, bz = op.beta
    U = np.zeros((N + 2, N + 2, N + 2))
    U[1:-1, 1:-1, 1:-1] = u.reshape(N, N, N)   # [k, j, i], x fastest
    c = U[1:-1, 1:-1, 1:-1]
    xm, xp = U[1:-1, 1:-1, :-2], U[1:-1, 1:-1, 2:]
    ym, yp = U[1:-1, :-2, 1:-1], U[1:-1, 2:, 1:-1]
    zm, zp = U[:-2, 1:-1, 1:-1], U[2:, 1:-1, 1:-1]
    Au = ((6.0 * c - xm - xp - ym - yp - zm - zp) / h**2
          + (bx * (xp - xm) + by * (yp - ym) + bz * (zp - zm)) / (2.0 * h) + op.mass * c)
    return Au.reshape(-1)


def _apply_vark2d(op: Operator, u):
    N = op.N
    h = 1.0 / (N + 1)
    bx = op.beta[0]
    K = op.kappa.reshape(N + 2, N + 2)        # nodes [j, i], 0..N+1
    U = np.zeros((N + 2, N + 2))
    U[1:-1, 1:-1] = u.reshape(N, N)
    c = U[1:-1, 1:-1]
    kc = K[1:-1, 1:-1]
    kw = 0.5 * (kc + K[1:-1, :-2])   # face between (i-1, j) and (i, j)
    ke = 0.5 * (kc + K[1:-1, 2:])
    ks = 0.5 * (kc + K[:-2, 1:-1])
    kn = 0.5 * (kc + K[2:, 1:-1])
    diff = (kw * (c - U[1:-1, :-2]) + ke * (c - U[1:-1, 2:])
            + ks * (c - U[:-2, 1:-1]) + kn * (c - U[2:, 1:-1])) / h**2
    conv = bx * (U[1:-1, 2:] - U[1:-1, :-2]) / (2.0 * h)
    return (diff + conv).reshape(-1)


def _grid_coo(N, dim):
    """Lexicographic index helper: returns a function (i, j[, k]) -> flat, 1-based coords."""
    if dim == 2:
        return lambda i, j: (j - 1) * N + (i - 1)
    return lambda i, j, k: (i - 1) + N * ((j - 1) + N * (k - 1))


def _assemble_cd2d(op: Operator):
    N = op.N
    h = 1.0 / (N + 1)
    bx = op.beta[0]
    idx = _grid_coo(N, 2)
    rows, cols, vals = [], [], []
    jj, ii = np.meshgrid(np.arange(1, N + 1), np.arange(1, N + 1), indexing="ij")
    ii, jj = ii.reshape(-1), jj.reshape(-1)
    me = idx(ii, jj)
    coefs = [((0, 0), 4.0 / h**2 + op.mass),
             ((-1, 0), -1.0 / h**2 - bx / (2 * h)), ((1, 0), -1.0 / h**2 + bx / (2 * h)),
             ((0, -1), -1.0 / h**2), ((0, 1), -1.0 / h**2)]
    for (di, dj), cval in coefs:
        ni, nj = ii + di, jj + dj
        ok = (ni >= 1) & (ni <= N) & (nj >= 1) & (nj <= N)
        rows.append(me[ok]); cols.append(idx(ni[ok], nj[ok])); vals.append(np.full(ok.sum(), cval))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N * N, N * N))


def _assemble_cd3d(op: Operator):
    N = op.N
    h = 1.0 / (N + 1)
    bx, by, bz = op.beta
    idx = _grid_coo(N, 3)
    kk, jj, ii = np.meshgrid(*(np.arange(1, N + 1),) * 3, indexing="ij")
    ii, jj, kk = ii.reshape(-1), jj.reshape(-1), kk.reshape(-1)
    me = idx(ii, jj, kk)
    d = -1.0 / h**2
    coefs = [((0, 0, 0), 6.0 / h**2 + op.mass),
             ((-1, 0, 0), d - bx / (2 * h)), ((1, 0, 0), d + bx / (2 * h)),
             ((0, -1, 0), d - by / (2 * h)), ((0, 1, 0), d + by / (2 * h)),
             ((0, 0, -1), d - bz / (2 * h)), ((0, 0, 1), d + bz / (2 * h))]
    rows, cols, vals = [], [], []
    for (di, dj, dk), cval in coefs:
        ni, nj, nk = ii + di, jj + dj, kk + dk
        ok = (ni >= 1) & (ni <= N) & (nj >= 1) & (nj <= N) & (nk >= 1) & (nk <= N)
        rows.append(me[ok]); cols.append(idx(ni[ok], nj[ok], nk[ok]))
        vals.append(np.full(ok.sum(), cval))
    n = N ** 3
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def _assemble_exp2d(op: Operator):
    """Entry by entry: row (i, j) holds a(i, j) (4, -1, -1, -1, -1) / h^2 for the diffusion and
    -+ b / (2h) for the convection towards the -/+ neighbour, plus c on the diagonal; the
    transpose is assembled as the transpose of that matrix."""
    N = op.N
    h = 1.0 / (N + 1)
    bx, by, gamma = op.beta
    idx = _grid_coo(N, 2)
    rows, cols, vals = [], [], []
    for j in range(1, N + 1):
        for i in range(1, N + 1):
            a = np.exp(gamma * (i * h) * (j * h))
            me = idx(i, j)
            rows.append(me); cols.append(me); vals.append(4.0 * a / h**2 + op.mass)
            for (di, dj, b) in ((-1, 0, -bx), (1, 0, bx), (0, -1, -by), (0, 1, by)):
                ni, nj = i + di, j + dj
                if 1 <= ni <= N and 1 <= nj <= N:
                    rows.append(me); cols.append(idx(ni, nj)); vals.append(-a / h**2 + b / (2 * h))
    M = sp.csr_matrix((vals, (rows, cols)), shape=(N * N, N * N))
    return M.T.tocsr() if op.transpose else M


def _assemble_vark2d(op: Operator):
    N = op.N
    h = 1.0 / (N + 1)
    bx = op.beta[0]
    K = op.kappa.reshape(N + 2, N + 2)
    idx = _grid_coo(N, 2)
    rows, cols, vals = [], [], []
    for j in range(1, N + 1):
        for i in range(1, N + 1):
            me = idx(i, j)
            diag = 0.0
            for (di, dj) in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                kf = 0.5 * (K[j, i] + K[j + dj, i + di])
                diag += kf / h**2
                cval = -kf / h**2 + di * bx / (2 * h)
                ni, nj = i + di, j + dj
                if 1 <= ni <= N and 1 <= nj <= N:
                    rows.append(me); cols.append(idx(ni, nj)); vals.append(cval)
            rows.append(me); cols.append(me); vals.append(diag)
    return sp.csr_matrix((vals, (rows, cols)), shape=(N * N, N * N))


# ----------------------------------------------------------------------------- lattice

def _axis(mu: int) -> int:
    # site index x0 + L(x1 + L(x2 + L x3)) -> numpy array [x3, x2, x1, x0]
    return 3 - mu


def _apply_u1(op: Operator, psi):
    L = op.N
    P = psi.reshape(L, L, L, L)
    out = (op.mass + 8.0) * P
    for mu in range(4):
        U = op.links[mu].reshape(L, L, L, L)
        ax = _axis(mu)
        fwd = np.roll(P, -1, axis=ax)                    # psi(x + mu)
        bwd = np.roll(np.conj(U) * P, 1, axis=ax)       # conj(U_mu(x - mu)) psi(x - mu)
        out = out - U * fwd - bwd
    return out.reshape(-1)


def lattice_shift_index(L: int, mu: int, sign: int) -> np.ndarray:
    """Flat index of x + sign*mu_hat for every site x (periodic)."""
    x = np.arange(L ** 4)
    c = [(x // L ** a) % L for a in range(4)]
    c[mu] = (c[mu] + sign) % L
    return c[0] + L * (c[1] + L * (c[2] + L * c[3]))


def _assemble_u1(op: Operator):
    L = op.N
    V = L ** 4
    x = np.arange(V)
    rows = [x]
    cols = [x]
    vals = [np.full(V, op.mass + 8.0, dtype=np.complex128)]
    for mu in range(4):
        xp = lattice_shift_index(L, mu, +1)
        xm = lattice_shift_index(L, mu, -1)
        rows += [x, x]
        cols += [xp, xm]
        vals += [-op.links[mu], -np.conj(op.links[mu][xm])]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(V, V))


# ----------------------------------------------------------------------------- coarse ops

def coarse_operator(op: Operator) -> Operator:
    """Coarse-grid operator of the two-grid method.

    Grids: the same PDE rediscretised at h_c = 2h (the paper's coarse problems are the
    fine PDE at a coarser h, Example 1 and Example 4); N = 2 N_c + 1 so the grids nest,
    and kappa is injected, kappa_c(I, J) = kappa(2I, 2J).
    The lattice coarse operator is the Galerkin product P^H A P and is built in
    oracle.transfer (it needs the block-transport prolongation P).
    """
    if op.kind == U1_4D:
        raise ValueError("use transfer.lattice_coarse_operator")
    if op.N % 2 != 1:
        raise ValueError("fine N must be odd so that the coarse grid nests")
    Nc = (op.N - 1) // 2
    kc = None
    if op.kind == VARK2D:
        K = op.kappa.reshape(op.N + 2, op.N + 2)
        kc = K[::2, ::2].reshape(-1).copy()
        assert kc.size == (Nc + 2) ** 2
    return Operator(op.kind, Nc, op.beta, kc, None, op.mass, transpose=op.transpose)


def cd2d_eigenvalues(N: int, beta: float) -> np.ndarray:
    """Closed-form eigenvalues of cd2d (centred convection in x only).

    With gamma = beta h / 2 and |gamma| < 1 the 1D operator tridiag(-1-gamma, 2, -1+gamma)/h^2
    is diagonally similar to the symmetric tridiag(-sqrt(1-gamma^2), 2, ...)/h^2, so
    lambda_pq = [4 - 2 sqrt(1 - gamma^2) cos(p pi h) - 2 cos(q pi h)] / h^2, p, q = 1..N.
    """
    h = 1.0 / (N + 1)
    g = beta * h / 2.0
    if abs(g) >= 1:
        raise ValueError("closed form needs |beta h / 2| < 1")
    p = np.arange(1, N + 1)
    ax = 2.0 - 2.0 * np.sqrt(1.0 - g * g) * np.cos(p * np.pi * h)
    ay = 2.0 - 2.0 * np.cos(p * np.pi * h)
    return np.sort((ax[:, None] + ay[None, :]).reshape(-1) / h**2)


def cd3d_eigenvalues(N: int, beta) -> np.ndarray:
    """Closed-form eigenvalues of cd3d: a sum of three 1D terms of the same form."""
    h = 1.0 / (N + 1)
    p = np.arange(1, N + 1)
    terms = []
    for b in beta:
        g = b * h / 2.0
        if abs(g) >= 1:
            raise ValueError("closed form needs |beta h / 2| < 1")
        terms.append(2.0 - 2.0 * np.sqrt(1.0 - g * g) * np.cos(p * np.pi * h))
    lam = terms[0][:, None, None] + terms[1][None, :, None] + terms[2][None, None, :]
    return np.sort(lam.reshape(-1) / h**2)


def free_lattice_eigenvalues(L: int, mass: float) -> np.ndarray:
    """Eigenvalues of u1_4d with all links 1: m + 8 - 2 sum_mu cos(2 pi n_mu / L) (Fourier)."""
    c = 2.0 * np.cos(2.0 * np.pi * np.arange(L) / L)
    s = (c[:, None, None, None] + c[None, :, None, None]
         + c[None, None, :, None] + c[None, None, None, :])
    return np.sort((mass + 8.0 - s).reshape(-1))


def lattice_tuned_mass(links: np.ndarray, L: int, lam_min: float = 1e-3,
                       iters: int = 200, seed: int = 0) -> float:
    """Mass m such that the smallest eigenvalue of u1_4d is lam_min.

    A = (m + 8) I - D with D the Hermitian hopping term, so lambda_min(A) = m + 8 -
    lambda_max(D).  lambda_max(D) is the top Ritz value of plain Lanczos on D (the
    extreme Ritz value converges without reorthogonalisation; loss of orthogonality only
    adds copies of it), then m = lambda_max(D) - 8 + lam_min.
    """
    op0 = Operator(U1_4D, L, links=links, mass=-8.0)    # apply = -D
    rng = np.random.default_rng(seed)
    V = L ** 4
    q = rng.standard_normal(V) + 1j * rng.standard_normal(V)
    q /= np.linalg.norm(q)
    qprev = np.zeros_like(q)
    alpha, betas = [], []
    b = 0.0
    for _ in range(iters):
        w = -op0.apply(q)
        a = np.vdot(q, w).real
        w = w - a * q - b * qprev
        alpha.append(a)
        b = np.linalg.norm(w)
        betas.append(b)
        if b == 0.0:
            break
        qprev, q = q, w / b
    T = np.diag(alpha) + np.diag(betas[:len(alpha) - 1], 1) + np.diag(betas[:len(alpha) - 1], -1)
    lam_max = np.linalg.eigvalsh(T)[-1]
    return float(lam_max - 8.0 + lam_min)
