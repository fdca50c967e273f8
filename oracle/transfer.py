"""Grid transfer between the coarse and fine problems, FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 3, phase 1: the coarse solution and the approximate eigenvectors are moved to
the fine grid.  The paper generally uses spline interpolation; this build uses bilinear
(2D), trilinear (3D) and 2^4 block transport (lattice) by default, and offers a
fourth-order cubic interpolation on the grids (below) as the stand-in for the splines.
Readings taken:

  * Nested vertex-centred grids: N = 2 N_c + 1; coarse node I sits on fine node 2I;
    coarse values beyond the grid (I = 0, N_c + 1) are the Dirichlet zero.
  * Fixed summation order, so that the result is reproducible bit for bit: pairs are
    summed along x first, then y, then z, and the weight (1/2 per interpolated axis) is
    applied last (a power of two, so it is exact).
  * Restriction for the coarse right-hand side: full weighting R = P^T / 2^d.
  * Lattice: blocks B(X) = {2X + delta, delta in {0,1}^4}; P[x, X] = (1/4) conj(W(x)),
    W(x) the product of the links along the path from the corner 2X to x that steps
    in mu = 0, 1, 2, 3 order.  P^H P = I, the coarse operator is P^H A P (Galerkin),
    and the construction is gauge covariant.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .operators import Operator, U1_4D, lattice_shift_index


def _pad2(uc, Nc):
    U = np.zeros((Nc + 2, Nc + 2))
    U[1:-1, 1:-1] = uc.reshape(Nc, Nc)
    return U


def prolong2d(uc: np.ndarray, Nc: int) -> np.ndarray:
    """Bilinear prolongation, coarse Nc^2 -> fine (2Nc+1)^2, x fastest."""
    N = 2 * Nc + 1
    C = _pad2(uc, Nc)                       # C[J, I], I, J in 0..Nc+1
    F = np.zeros((N + 2, N + 2))            # F[j, i], i, j in 0..N+1
    # coincident points
    F[2:N + 1:2, 2:N + 1:2] = C[1:Nc + 1, 1:Nc + 1]
    # x-edge points (2I+1, 2J): I = 0..Nc, J = 1..Nc
    F[2:N + 1:2, 1:N + 1:2] = 0.5 * (C[1:Nc + 1, 0:Nc + 1] + C[1:Nc + 1, 1:Nc + 2])
    # y-edge points (2I, 2J+1)
    F[1:N + 1:2, 2:N + 1:2] = 0.5 * (C[0:Nc + 1, 1:Nc + 1] + C[1:Nc + 2, 1:Nc + 1])
    # cell centres (2I+1, 2J+1): x pairs first, then y
    F[1:N + 1:2, 1:N + 1:2] = 0.25 * ((C[0:Nc + 1, 0:Nc + 1] + C[0:Nc + 1, 1:Nc + 2])
                                      + (C[1:Nc + 2, 0:Nc + 1] + C[1:Nc + 2, 1:Nc + 2]))
    return F[1:-1, 1:-1].reshape(-1).copy()


def prolong3d(uc: np.ndarray, Nc: int) -> np.ndarray:
    """Trilinear prolongation, coarse Nc^3 -> fine (2Nc+1)^3, x fastest.

    Written point by point over the 8 parity classes: for a fine point with parities
    (px, py, pz) the corners are summed as a pairwise tree in x, then y, then z."""
    N = 2 * Nc + 1
    C = np.zeros((Nc + 2,) * 3)
    C[1:-1, 1:-1, 1:-1] = uc.reshape(Nc, Nc, Nc)    # [K, J, I]
    F = np.zeros((N,) * 3)                           # [k-1, j-1, i-1]

    def sl(p):
        # fine 1-based coords with parity p: even -> 2I (I = 1..Nc), odd -> 2I+1 (I = 0..Nc)
        # returns (fine slice 0-based, coarse low-corner slice)
        if p == 0:
            return slice(1, N, 2), slice(1, Nc + 1)
        return slice(0, N, 2), slice(0, Nc + 1)

    for pz in (0, 1):
        fz, cz = sl(pz)
        for py in (0, 1):
            fy, cy = sl(py)
            for px in (0, 1):
                fx, cx = sl(px)

                def corner(dx, dy, dz):
                    return C[cz.start + dz:cz.stop + dz, cy.start + dy:cy.stop + dy,
                             cx.start + dx:cx.stop + dx]

                def xsum(dy, dz):
                    return corner(0, dy, dz) + corner(1, dy, dz) if px else corner(0, dy, dz)

                def ysum(dz):
                    return xsum(0, dz) + xsum(1, dz) if py else xsum(0, dz)

                tot = ysum(0) + ysum(1) if pz else ysum(0)
                w = 0.5 ** (px + py + pz)
                F[fz, fy, fx] = w * tot
    return F.reshape(-1).copy()


# ----------------------------------------------------------------------------- cubic
# Fourth-order interpolation standing in for the paper's spline interpolation (Section 3,
# phase 1: the paper generally uses splines to move the eigenvectors).  Readings taken:
#
#  * a new fine point halfway between coarse nodes a and a + 1 takes the cubic through the
#    four coarse nodes a - 1 .. a + 2: weights (-1, 9, 9, -1) / 16 (exact for cubics);
#    fine points on coarse nodes copy them;
#  * beyond the Dirichlet boundary the grid function is continued oddly: node 0 and node
#    N_c + 1 are the boundary zeros, node -1 is -u(1) and node N_c + 2 is -u(N_c), so
#    every mode sin(p pi x) is continued exactly;
#  * tensor product, axes in the order x, y, z; each 4-term sum is evaluated as
#    ((w0 v0 + w1 v1) + w2 v2) + w3 v3 with separate rounded products (the weights are
#    exact binary fractions), so the result is reproducible bit for bit.

CUBIC_W = (-0.0625, 0.5625, 0.5625, -0.0625)


def _cubic_axis(U: np.ndarray) -> np.ndarray:
    """Interpolate along the last axis: (..., Nc) -> (..., 2 Nc + 1)."""
    Nc = U.shape[-1]
    z = np.zeros_like(U[..., :1])
    # padded nodes -1, 0, 1..Nc, Nc+1, Nc+2 at positions 0..Nc+3
    P = np.concatenate([-U[..., :1], z, U, z, -U[..., -1:]], axis=-1)
    out = np.empty(U.shape[:-1] + (2 * Nc + 1,))
    out[..., 1::2] = U                           # fine index 2I (1-based) = coarse node I
    a = np.arange(0, Nc + 1)                     # fine index 2a + 1 lies between nodes a, a + 1
    v = [P[..., a + q] for q in range(4)]        # nodes a - 1 .. a + 2 sit at positions a .. a + 3
    w = CUBIC_W
    out[..., 0::2] = ((w[0] * v[0] + w[1] * v[1]) + w[2] * v[2]) + w[3] * v[3]
    return out


def prolong2d_cubic(uc: np.ndarray, Nc: int) -> np.ndarray:
    """Cubic prolongation, coarse Nc^2 -> fine (2Nc+1)^2, x fastest (x first, then y)."""
    U = uc.reshape(Nc, Nc)                       # [J, I]
    T = _cubic_axis(U)                           # [J, i]
    F = _cubic_axis(T.T).T                       # [j, i]
    return np.ascontiguousarray(F).reshape(-1)


def prolong3d_cubic(uc: np.ndarray, Nc: int) -> np.ndarray:
    """Cubic prolongation, coarse Nc^3 -> fine (2Nc+1)^3, x fastest (x, then y, then z)."""
    U = uc.reshape(Nc, Nc, Nc)                   # [K, J, I]
    T = _cubic_axis(U)                           # [K, J, i]
    T = np.swapaxes(_cubic_axis(np.swapaxes(T, 1, 2)), 1, 2)       # [K, j, i]
    F = np.swapaxes(_cubic_axis(np.swapaxes(T, 0, 2)), 0, 2)       # [k, j, i]
    return np.ascontiguousarray(F).reshape(-1)


def prolongation_matrix(Nc: int, dim: int):
    """Sparse P (n_fine x n_coarse) built entry by entry from the interpolation weights
    (an independent statement of the same map, used to check prolong2d/3d)."""
    N = 2 * Nc + 1
    rows, cols, vals = [], [], []
    w1 = {0: [(0, 1.0)], 1: [(0, 0.5), (1, 0.5)]}     # parity -> (offset, weight) from low corner
    rng = range(1, N + 1)
    if dim == 2:
        for j in rng:
            for i in rng:
                f = (j - 1) * N + (i - 1)
                for oy, wy in w1[j % 2]:
                    for ox, wx in w1[i % 2]:
                        I, J = i // 2 + ox, j // 2 + oy
                        if 1 <= I <= Nc and 1 <= J <= Nc:
                            rows.append(f); cols.append((J - 1) * Nc + (I - 1)); vals.append(wx * wy)
        return sp.csr_matrix((vals, (rows, cols)), shape=(N * N, Nc * Nc))
    for k in rng:
        for j in rng:
            for i in rng:
                f = (i - 1) + N * ((j - 1) + N * (k - 1))
                for oz, wz in w1[k % 2]:
                    for oy, wy in w1[j % 2]:
                        for ox, wx in w1[i % 2]:
                            I, J, K = i // 2 + ox, j // 2 + oy, k // 2 + oz
                            if 1 <= I <= Nc and 1 <= J <= Nc and 1 <= K <= Nc:
                                rows.append(f)
                                cols.append((I - 1) + Nc * ((J - 1) + Nc * (K - 1)))
                                vals.append(wx * wy * wz)
    return sp.csr_matrix((vals, (rows, cols)), shape=(N ** 3, Nc ** 3))


def restrict(uf: np.ndarray, N: int, dim: int) -> np.ndarray:
    """Full-weighting restriction R = P^T / 2^dim (fine N -> coarse (N-1)/2)."""
    Nc = (N - 1) // 2
    P = prolongation_matrix(Nc, dim)
    return (P.T @ uf) / 2.0 ** dim


def restrict_stencil(uf: np.ndarray, N: int, dim: int) -> np.ndarray:
    """The same full weighting written as its stencil (vectorised, for large grids): the
    coarse value at node I is 2^-dim times the sum over the fine nodes 2I + o,
    o in {-1, 0, 1}^dim, of u(2I + o) times prod_axes w(o_a), w(0) = 1, w(+-1) = 1/2 -- the
    transpose of the bilinear / trilinear weights (fine values beyond the grid are zero)."""
    Nc = (N - 1) // 2
    F = np.zeros((N + 2,) * dim)
    F[(slice(1, N + 1),) * dim] = uf.reshape((N,) * dim)     # [.., j, i], 0..N+1 with zero borders
    out = np.zeros((Nc,) * dim)
    w = {-1: 0.5, 0: 1.0, 1: 0.5}
    for offs in np.ndindex(*(3,) * dim):
        o = [v - 1 for v in offs]
        wt = np.prod([w[v] for v in o])
        # fine index 2I + o for I = 1..Nc  ->  padded index 2I + o
        sl = tuple(slice(2 + v, 2 * Nc + 1 + v, 2) for v in o)
        out += wt * F[sl]
    return out.reshape(-1) / 2.0 ** dim


# ----------------------------------------------------------------------------- lattice

def lattice_prolongation(links: np.ndarray, L: int):
    """Block-transport prolongation P (L^4 x (L/2)^4), complex128, sparse."""
    Lc = L // 2
    Vc = Lc ** 4
    rows, cols, vals = [], [], []
    X = np.arange(Vc)
    Xc = [(X // Lc ** a) % Lc for a in range(4)]
    for d in range(16):
        delta = [(d >> a) & 1 for a in range(4)]
        y = [2 * Xc[a] for a in range(4)]               # path position, start at corner 2X
        W = np.ones(Vc, dtype=np.complex128)
        for mu in range(4):
            if delta[mu]:
                site = y[0] + L * (y[1] + L * (y[2] + L * y[3]))
                W = W * links[mu][site]
                y[mu] = y[mu] + 1
        x = y[0] + L * (y[1] + L * (y[2] + L * y[3]))
        rows.append(x); cols.append(X); vals.append(0.25 * np.conj(W))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(L ** 4, Vc))


def lattice_coarse_stencil(op: Operator):
    """Galerkin coarse operator A_c = P^H A P of the lattice, as the sparse product and
    as its 9-point stencil: (diag[X], fwd[mu][X] = A_c[X, X+mu], bwd[mu][X] = A_c[X, X-mu])."""
    assert op.kind == U1_4D
    L = op.N
    Lc = L // 2
    P = lattice_prolongation(op.links, L)
    Ac = (P.conj().T @ op.sparse() @ P).tocsr()
    Vc = Lc ** 4
    X = np.arange(Vc)
    diag = np.asarray(Ac[X, X]).reshape(-1)
    fwd = np.zeros((4, Vc), dtype=np.complex128)
    bwd = np.zeros((4, Vc), dtype=np.complex128)
    for mu in range(4):
        fwd[mu] = np.asarray(Ac[X, lattice_shift_index(Lc, mu, +1)]).reshape(-1)
        bwd[mu] = np.asarray(Ac[X, lattice_shift_index(Lc, mu, -1)]).reshape(-1)
    return Ac, P, diag, fwd, bwd


def apply_lattice_coarse(diag, fwd, bwd, Lc, psi):
    """Apply the 9-point coarse stencil (used to check it against the sparse A_c)."""
    out = diag * psi
    for mu in range(4):
        out = out + fwd[mu] * psi[lattice_shift_index(Lc, mu, +1)]
        out = out + bwd[mu] * psi[lattice_shift_index(Lc, mu, -1)]
    return out
