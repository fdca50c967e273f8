"""Pins of the oracle's operators and grid transfer to facts the paper and mathematics fix.

- closed-form eigenvalues of the centred convection-diffusion operator (diagonally
  similar to a symmetric one when |beta h / 2| < 1), checked against LAPACK eig of the
  independently assembled sparse matrix;
- the free-field lattice spectrum (Fourier), Hermiticity and gauge covariance;
- A^T = A(kappa, -beta) at matrix level;
- bilinear/trilinear prolongation reproduces linear functions; its point formulas agree
  with an entry-by-entry sparse P; P^H P = I for the lattice block transport, and the
  Galerkin coarse operator of the free field has the closed form (m + 4) I - 1/2 hops.
"""
import numpy as np
import pytest

import tg_inputs as gi
from oracle import transfer
from oracle.operators import (CD2D, CD3D, U1_4D, VARK2D, Operator, cd2d_eigenvalues,
                              cd3d_eigenvalues, coarse_operator, free_lattice_eigenvalues,
                              lattice_shift_index)


@pytest.mark.parametrize("N,beta", [(9, 3.0), (15, 1.0), (7, -5.0)])
def test_cd2d_closed_form_spectrum(N, beta):
    op = Operator(CD2D, N, (beta,))
    lam = np.sort(np.linalg.eigvals(op.sparse().toarray()).real)
    ref = cd2d_eigenvalues(N, beta)
    assert np.max(np.abs(lam - ref)) / ref.max() < 1e-13


def test_cd3d_closed_form_spectrum():
    op = Operator(CD3D, 5, (2.0, 1.0, 0.5))
    lam = np.sort(np.linalg.eigvals(op.sparse().toarray()).real)
    ref = cd3d_eigenvalues(5, (2.0, 1.0, 0.5))
    assert np.max(np.abs(lam - ref)) / ref.max() < 1e-13


def test_cfg_sizes_smallest_eigenvalue():
    # 127^2, beta = 1: the continuum operator -Lap + beta d/dx is similar to
    # -Lap + beta^2/4, whose smallest eigenvalue on the unit square is 2 pi^2 + beta^2/4
    lmin = cd2d_eigenvalues(127, 1.0)[0]
    assert abs(lmin - 19.988) < 1e-3
    assert abs(lmin - (2 * np.pi ** 2 + 0.25)) / lmin < 1e-4


@pytest.mark.parametrize("kind,N,beta", [(CD2D, 11, (2.0,)), (CD3D, 5, (2.0, 1.0, 0.5))])
def test_matrix_free_equals_assembled(kind, N, beta):
    op = Operator(kind, N, beta)
    u = gi.random_dense(op.n, 1)
    y = op.apply(u)
    assert np.max(np.abs(y - op.sparse() @ u)) <= 1e-14 * np.max(np.abs(y))


def test_vark2d_assembled_and_special_case():
    N = 9
    kap = gi.kappa_grf(N, 0)
    op = Operator(VARK2D, N, (1.0,), kap)
    u = gi.random_dense(op.n, 2)
    y = op.apply(u)
    assert np.max(np.abs(y - op.sparse() @ u)) <= 1e-14 * np.max(np.abs(y))
    # kappa == 1 reduces to the constant-coefficient operator
    one = Operator(VARK2D, N, (1.0,), np.ones((N + 2) ** 2))
    assert np.max(np.abs(one.apply(u) - Operator(CD2D, N, (1.0,)).apply(u))) <= 1e-12 * np.max(np.abs(y))


@pytest.mark.parametrize("kind", [CD2D, CD3D, VARK2D])
def test_transpose_is_beta_negated(kind):
    N = 7
    beta = (1.5,) if kind != CD3D else (2.0, 1.0, 0.5)
    kap = gi.kappa_grf(N, 1) if kind == VARK2D else None
    op = Operator(kind, N, beta, kap)
    diff = (op.sparse().T - op.transposed().sparse()).toarray()
    assert np.max(np.abs(diff)) == 0.0


def test_lattice_free_field_spectrum():
    L, m = 4, 0.3
    op = Operator(U1_4D, L, links=np.ones((4, L ** 4), dtype=np.complex128), mass=m)
    lam = np.linalg.eigvalsh(op.sparse().toarray())
    assert np.max(np.abs(np.sort(lam) - free_lattice_eigenvalues(L, m))) < 1e-12


def test_lattice_hermitian_and_gauge_covariant():
    L = 4
    links = gi.u1_links(L, 3)
    op = Operator(U1_4D, L, links=links, mass=0.2)
    A = op.sparse().toarray()
    assert np.max(np.abs(A - A.conj().T)) == 0.0
    psi = gi.random_dense(L ** 4, 4) + 1j * gi.random_dense(L ** 4, 5)
    assert np.max(np.abs(op.apply(psi) - A @ psi)) < 1e-13
    g = np.exp(1j * gi.random_dense(L ** 4, 6))
    links2 = np.stack([g * links[mu] * np.conj(g[lattice_shift_index(L, mu, +1)]) for mu in range(4)])
    op2 = Operator(U1_4D, L, links=links2, mass=0.2)
    assert np.max(np.abs(op2.apply(g * psi) - g * op.apply(psi))) < 1e-12


def _linear(xs, ys, zs=None):
    f = 0.3 + 1.7 * xs - 0.9 * ys
    return f if zs is None else f + 0.4 * zs


def test_prolong2d_reproduces_linear_and_matches_sparse():
    Nc = 7
    N = 2 * Nc + 1
    hc, h = 1.0 / (Nc + 1), 1.0 / (N + 1)
    J, I = np.meshgrid(np.arange(1, Nc + 1), np.arange(1, Nc + 1), indexing="ij")
    uc = _linear(I * hc, J * hc).reshape(-1)
    uf = transfer.prolong2d(uc, Nc).reshape(N, N)
    j, i = np.meshgrid(np.arange(1, N + 1), np.arange(1, N + 1), indexing="ij")
    exact = _linear(i * h, j * h)
    inner = (i >= 2) & (i <= N - 1) & (j >= 2) & (j <= N - 1)   # stencil clear of the boundary
    assert np.max(np.abs(uf - exact)[inner]) < 1e-14
    w = gi.random_dense(Nc * Nc, 3)
    assert np.max(np.abs(transfer.prolong2d(w, Nc) - transfer.prolongation_matrix(Nc, 2) @ w)) < 1e-15


def _cubic_matrix_1d(Nc):
    """The 1D cubic interpolation written entry by entry from its rule: fine node 2I copies
    coarse node I; fine node 2a + 1 takes (-1, 9, 9, -1)/16 of nodes a-1 .. a+2, where
    nodes 0 and Nc+1 are zero and nodes -1, Nc+2 are -u(1), -u(Nc) (odd continuation)."""
    N = 2 * Nc + 1
    P = np.zeros((N, Nc))
    for i in range(1, N + 1):
        if i % 2 == 0:
            P[i - 1, i // 2 - 1] = 1.0
            continue
        a = (i - 1) // 2
        for node, w in zip(range(a - 1, a + 3), (-1 / 16, 9 / 16, 9 / 16, -1 / 16)):
            if node == -1:
                P[i - 1, 0] -= w
            elif node == Nc + 2:
                P[i - 1, Nc - 1] -= w
            elif 1 <= node <= Nc:
                P[i - 1, node - 1] += w
    return P


def test_cubic_prolongation_pins():
    """Cubic prolongation (the stand-in for the paper's splines): (1) fine nodes on coarse
    nodes copy them bit for bit; (2) it reproduces cubic polynomials wherever its stencil
    stays inside the grid; (3) it equals the entry-by-entry Kronecker product of the 1D
    rule; (4) on the Dirichlet modes sin(p pi x) sin(q pi y) the error is fourth order (the
    odd continuation is exact for them, boundary rows included) and within the Lagrange
    remainder bound of the 4-point cubic at a midpoint, 9/16 h^4 |f''''| / 24 per axis."""
    rng = np.random.default_rng(11)
    Nc = 9
    N = 2 * Nc + 1
    uc = rng.standard_normal(Nc * Nc)
    uf = transfer.prolong2d_cubic(uc, Nc).reshape(N, N)
    assert np.array_equal(uf[1::2, 1::2], uc.reshape(Nc, Nc))
    P1 = _cubic_matrix_1d(Nc)
    assert np.max(np.abs(uf.reshape(-1) - np.kron(P1, P1) @ uc)) < 1e-14
    uc3 = rng.standard_normal(5 ** 3)
    P5 = _cubic_matrix_1d(5)
    assert np.max(np.abs(transfer.prolong3d_cubic(uc3, 5) - np.kron(P5, np.kron(P5, P5)) @ uc3)) < 1e-14
    # cubic polynomials
    hc, h = 1.0 / (Nc + 1), 1.0 / (N + 1)

    def cub(x, y):
        return 0.2 - x + 2.0 * x ** 3 - 0.5 * x ** 2 * y + 1.5 * y ** 3 + 0.7 * x * y ** 2

    J, I = np.meshgrid(np.arange(1, Nc + 1), np.arange(1, Nc + 1), indexing="ij")
    ufc = transfer.prolong2d_cubic(cub(I * hc, J * hc).reshape(-1), Nc).reshape(N, N)
    j, i = np.meshgrid(np.arange(1, N + 1), np.arange(1, N + 1), indexing="ij")
    inner = (i >= 4) & (i <= N - 3) & (j >= 4) & (j <= N - 3)   # every stencil node in 1..Nc
    assert inner.sum() > 0
    assert np.max(np.abs(ufc - cub(i * h, j * h))[inner]) < 1e-13
    # fourth order on a Dirichlet mode, boundary rows included
    p, q = 3, 2
    errs = []
    for Ncs in (15, 31, 63):
        Ns = 2 * Ncs + 1
        xc = np.arange(1, Ncs + 1) / (Ncs + 1)
        xf = np.arange(1, Ns + 1) / (Ns + 1)
        mode_c = np.outer(np.sin(q * np.pi * xc), np.sin(p * np.pi * xc)).reshape(-1)
        mode_f = np.outer(np.sin(q * np.pi * xf), np.sin(p * np.pi * xf))
        e = np.max(np.abs(transfer.prolong2d_cubic(mode_c, Ncs).reshape(Ns, Ns) - mode_f))
        bound = (9 / 16) / 24 * (1.0 / (Ncs + 1)) ** 4 * ((p * np.pi) ** 4 + (q * np.pi) ** 4) * (1 + 1 / 8)
        assert e <= bound
        errs.append(e)
    assert 12.0 < errs[0] / errs[1] < 20.0 and 12.0 < errs[1] / errs[2] < 20.0
    # bilinear is only second order on the same mode
    Ncs = 31
    xc = np.arange(1, Ncs + 1) / (Ncs + 1)
    xf = np.arange(1, 2 * Ncs + 2) / (2 * Ncs + 2)
    mode_c = np.outer(np.sin(q * np.pi * xc), np.sin(p * np.pi * xc)).reshape(-1)
    mode_f = np.outer(np.sin(q * np.pi * xf), np.sin(p * np.pi * xf)).reshape(-1)
    assert np.max(np.abs(transfer.prolong2d(mode_c, Ncs) - mode_f)) > 20 * errs[1]


def test_prolong3d_reproduces_linear_and_matches_sparse():
    Nc = 4
    N = 2 * Nc + 1
    hc, h = 1.0 / (Nc + 1), 1.0 / (N + 1)
    K, J, I = np.meshgrid(*(np.arange(1, Nc + 1),) * 3, indexing="ij")
    uc = _linear(I * hc, J * hc, K * hc).reshape(-1)
    uf = transfer.prolong3d(uc, Nc).reshape(N, N, N)
    k, j, i = np.meshgrid(*(np.arange(1, N + 1),) * 3, indexing="ij")
    exact = _linear(i * h, j * h, k * h)
    inner = (i >= 2) & (i <= N - 1) & (j >= 2) & (j <= N - 1) & (k >= 2) & (k <= N - 1)
    assert np.max(np.abs(uf - exact)[inner]) < 1e-14
    w = gi.random_dense(Nc ** 3, 3)
    assert np.max(np.abs(transfer.prolong3d(w, Nc) - transfer.prolongation_matrix(Nc, 3) @ w)) < 1e-15


def test_full_weighting_of_constant():
    N = 15
    uf = np.ones(N * N)
    uc = transfer.restrict(uf, N, 2).reshape(7, 7)
    assert np.allclose(uc[1:-1, 1:-1], 1.0, atol=1e-15)
    uc3 = transfer.restrict(np.ones(9 ** 3), 9, 3).reshape(4, 4, 4)
    assert np.allclose(uc3[1:-1, 1:-1, 1:-1], 1.0, atol=1e-15)


def test_coarse_rediscretisation():
    op = Operator(VARK2D, 9, (1.0,), gi.kappa_grf(9, 2))
    opc = coarse_operator(op)
    assert opc.N == 4
    K = op.kappa.reshape(11, 11)
    assert np.array_equal(opc.kappa.reshape(6, 6), K[::2, ::2])


def test_lattice_block_transport():
    L = 8
    links = gi.u1_links(L, 0)
    op = Operator(U1_4D, L, links=links, mass=0.1)
    Ac, P, diag, fwd, bwd = transfer.lattice_coarse_stencil(op)
    assert np.max(np.abs((P.conj().T @ P).toarray() - np.eye(P.shape[1]))) < 1e-15
    D = Ac - Ac.conj().T
    assert abs(D).max() < 1e-14
    psi = gi.random_dense(4 ** 4, 1) + 1j * gi.random_dense(4 ** 4, 2)
    assert np.max(np.abs(transfer.apply_lattice_coarse(diag, fwd, bwd, 4, psi) - Ac @ psi)) < 1e-13
    assert Ac.nnz <= 9 * 4 ** 4


def test_lattice_coarse_free_field_closed_form():
    L, m = 8, 0.25
    op = Operator(U1_4D, L, links=np.ones((4, L ** 4), dtype=np.complex128), mass=m)
    _, _, diag, fwd, bwd = transfer.lattice_coarse_stencil(op)
    assert np.allclose(diag, m + 4.0, atol=1e-14)
    assert np.allclose(fwd, -0.5, atol=1e-14) and np.allclose(bwd, -0.5, atol=1e-14)


def test_lattice_coarse_gauge_covariant():
    L = 8
    links = gi.u1_links(L, 4)
    g = np.exp(1j * gi.random_dense(L ** 4, 7))
    links2 = np.stack([g * links[mu] * np.conj(g[lattice_shift_index(L, mu, +1)]) for mu in range(4)])
    Ac1 = transfer.lattice_coarse_stencil(Operator(U1_4D, L, links=links, mass=0.1))[0]
    Ac2 = transfer.lattice_coarse_stencil(Operator(U1_4D, L, links=links2, mass=0.1))[0]
    Lc = L // 2
    X = np.arange(Lc ** 4)
    Xc = [(X // Lc ** a) % Lc for a in range(4)]
    gc = g[2 * Xc[0] + L * (2 * Xc[1] + L * (2 * Xc[2] + L * 2 * Xc[3]))]
    import scipy.sparse as sp
    G = sp.diags(gc)
    assert abs(Ac2 - G @ Ac1 @ G.conj()).max() < 1e-13


def _dense_of(op):
    """The operator's dense matrix, column by column from its matrix-free apply."""
    n = op.n
    A = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[j] = 1.0
        A[:, j] = op.apply(e)
        e[j] = 0.0
    return A


def test_lattice_tuned_mass_free_field():
    """Free field (theta = 0): the hopping term's largest eigenvalue is 8 by Fourier
    (2 sum_mu cos 0), so the mass that puts lambda_min at 1e-3 is exactly 1e-3."""
    from oracle.operators import lattice_tuned_mass
    L = 4
    m = lattice_tuned_mass(np.ones((4, L ** 4), dtype=np.complex128), L, lam_min=1e-3)
    assert abs(m - 1e-3) < 1e-9


@pytest.mark.parametrize("seed", [0, 5])
def test_lattice_tuned_mass_random_field(seed):
    """On a random U(1) field the tuned mass makes the smallest eigenvalue of the dense
    Hermitian matrix (LAPACK eigvalsh) equal to the requested 1e-3."""
    from oracle.operators import lattice_tuned_mass
    L = 4
    links = gi.u1_links(L, seed)
    m = lattice_tuned_mass(links, L, lam_min=1e-3)
    lam = np.linalg.eigvalsh(_dense_of(Operator(U1_4D, L, links=links, mass=m)))
    assert abs(lam[0] - 1e-3) < 1e-9


@pytest.mark.parametrize("N,dim", [(15, 2), (9, 3), (31, 2)])
def test_restrict_stencil_equals_sparse_transpose(N, dim):
    """The vectorised full-weighting stencil is the transpose of the entry-by-entry sparse
    prolongation divided by 2^dim."""
    u = gi.random_dense(N ** dim, 9)
    a = transfer.restrict(u, N, dim)
    b = transfer.restrict_stencil(u, N, dim)
    assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(a))


def test_reaction_shift_closed_form():
    """cd2d with the reaction term c u (Example 4's Helmholtz form): the spectrum is the
    closed-form convection-diffusion spectrum shifted by c (LAPACK eig of the assembled
    matrix), and the shift survives transposition and coarsening."""
    from oracle.operators import cd2d_eigenvalues
    N, beta, c = 9, 3.0, -700.0
    op = Operator(CD2D, N, (beta,), mass=c)
    lam = np.sort(np.linalg.eigvals(op.sparse().toarray()).real)
    assert np.max(np.abs(lam - (cd2d_eigenvalues(N, beta) + c))) <= 1e-10 * np.max(np.abs(lam))
    u = gi.random_dense(op.n, 3)
    assert np.allclose(op.apply(u), op.sparse() @ u, rtol=1e-13, atol=1e-10)
    assert np.allclose(op.transposed().apply(u), op.sparse().T @ u, rtol=1e-13, atol=1e-10)
    assert coarse_operator(op).mass == c


def test_exp2d_without_exponent_closed_form():
    """Example 1's operator with gamma = 0 is -Lap + bx d_x + by d_y, diagonally similar to a
    symmetric matrix when |b h / 2| < 1 in both directions: its eigenvalues are
    [4 - 2 sqrt(1 - gx^2) cos(p pi h) - 2 sqrt(1 - gy^2) cos(q pi h)] / h^2, gx = bx h / 2."""
    from oracle.operators import EXP2D
    N, bx, by = 9, 3.0, -5.0
    h = 1.0 / (N + 1)
    p = np.arange(1, N + 1)
    tx = 2 - 2 * np.sqrt(1 - (bx * h / 2) ** 2) * np.cos(p * np.pi * h)
    ty = 2 - 2 * np.sqrt(1 - (by * h / 2) ** 2) * np.cos(p * np.pi * h)
    closed = np.sort((tx[:, None] + ty[None, :]).reshape(-1) / h**2)
    op = Operator(EXP2D, N, (bx, by, 0.0))
    lam = np.sort(np.linalg.eigvals(op.sparse().toarray()).real)
    assert np.max(np.abs(lam - closed)) <= 1e-10 * closed[-1]


@pytest.mark.parametrize("transpose", [False, True])
def test_exp2d_matrix_free_equals_assembled(transpose):
    from oracle.operators import EXP2D
    op = Operator(EXP2D, 15, (40.0, 40.0, 5.0), mass=-3.0)
    if transpose:
        A = op.sparse().T
        op = op.transposed()
    else:
        A = op.sparse()
    u = gi.random_dense(op.n, 4)
    y = op.apply(u)
    assert np.max(np.abs(y - A @ u)) <= 1e-12 * np.max(np.abs(y))
    c = coarse_operator(op)
    assert c.N == 7 and c.beta == op.beta and c.transpose == op.transpose


@pytest.mark.parametrize("kind", ["exp2d", "helmholtz"])
def test_continuum_limit(kind):
    """Applied to samples of a smooth u with zero boundary values, the discrete operator
    approaches the differential operator at the nodes with O(h^2) error (centred
    differences): -exp(5xy) Lap u + 40 u_x + 40 u_y (Example 1) and -Lap u - 100^2 u
    (Example 4), u = sin(pi x) sin(2 pi y), derivatives by hand."""
    from oracle.operators import EXP2D
    errs = []
    for N in (63, 127, 255):
        h = 1.0 / (N + 1)
        t = np.arange(1, N + 1) * h
        Y, X = np.meshgrid(t, t, indexing="ij")            # [j, i]
        u = np.sin(np.pi * X) * np.sin(2 * np.pi * Y)
        lap = -5 * np.pi ** 2 * u
        ux = np.pi * np.cos(np.pi * X) * np.sin(2 * np.pi * Y)
        uy = 2 * np.pi * np.sin(np.pi * X) * np.cos(2 * np.pi * Y)
        if kind == "exp2d":
            op = Operator(EXP2D, N, (40.0, 40.0, 5.0))
            exact = -np.exp(5 * X * Y) * lap + 40 * ux + 40 * uy
        else:
            op = Operator(CD2D, N, (0.0,), mass=-1e4)
            exact = -lap - 1e4 * u
        errs.append(np.max(np.abs(op.apply(u.reshape(-1)) - exact.reshape(-1))) / np.max(np.abs(exact)))
    assert errs[-1] < 1e-3
    for e0, e1 in zip(errs, errs[1:]):
        assert 3.5 < e0 / e1 < 4.5, errs
