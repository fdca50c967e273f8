"""Pins of the oracle's projections, BiCGStab, GMRES, GMRES-DR, two-grid driver and adjoint.

Each test checks the oracle against something other than itself:
  - projection invariants stated with the Section 2.2 projections (Galerkin: V^T r = 0;
    MinRes: (AV)^T r = 0 and ||r|| cannot grow), and exact eigenvectors removing their
    components;
  - brute force: dense LU solutions on <= 15^2 / 7^3 grids;
  - textbook special cases: A = lambda I converges in one BiCGStab half step; GMRES(n)
    on an n x n system is exact; one GMRES-DR cycle is GMRES(m);
  - the defining Petrov-Galerkin property of harmonic Ritz pairs (A y - theta y is
    orthogonal to A V_m), computed with the actual vectors;
  - harmonic Ritz values converge to the closed-form eigenvalues of the operator;
  - the Section 4.1 cycle tolerance: cycles meeting the first criterion reach rtol
    exactly at icyc = ncyc; the second criterion bounds progress to icyc/ncyc of the way;
  - adjoint gradient against central finite differences of direct solves.
Parity unpinned: iteration counts (they depend on rounding and on MATLAB internals).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import tg_inputs as gi
from oracle import adjoint, krylov, twogrid
from oracle.gmresdr import gmresdr, harmonic_ritz, select_k, eigen_residuals, arnoldi_extend
from oracle.operators import CD2D, CD3D, U1_4D, VARK2D, Operator, cd2d_eigenvalues


def _dense_solve(op, b):
    return np.linalg.solve(op.sparse().toarray(), b)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_minres_projection_invariants():
    op = Operator(CD2D, 15, (2.0,))
    Y = gi.random_dense((op.n, 6), 1)
    defl = krylov.make_deflation(op.apply, Y, "minres")
    b = gi.rhs(op.n, 0)
    x = gi.random_dense(op.n, 2)
    r = b - op.apply(x)
    x2, r2 = krylov.minres_project(defl, x, r)
    scale = np.linalg.norm(defl.AY) * np.linalg.norm(r)
    assert np.max(np.abs(defl.AY.T @ r2)) < 1e-13 * scale
    assert np.linalg.norm(r2) <= np.linalg.norm(r)
    assert _rel(r2, b - op.apply(x2)) < 1e-12


def test_galerkin_projection_invariants():
    op = Operator(CD2D, 15, (2.0,))
    Y = gi.random_dense((op.n, 6), 3)
    defl = krylov.make_deflation(op.apply, Y, "galerkin")
    b = gi.rhs(op.n, 1)
    x = np.zeros(op.n)
    x2, r2 = krylov.galerkin_project(defl, x, b.copy())
    assert np.max(np.abs(Y.T @ r2)) < 1e-12 * np.linalg.norm(Y) * np.linalg.norm(b)
    assert _rel(r2, b - op.apply(x2)) < 1e-12


def test_projection_with_exact_eigenvectors():
    op = Operator(CD2D, 11, (1.0,))
    lam, W = np.linalg.eig(op.sparse().toarray())
    idx = np.argsort(lam.real)[:5]
    Y = W[:, idx].real
    b = gi.rhs(op.n, 4)
    defl = krylov.make_deflation(op.apply, Y, "minres")
    _, r2 = krylov.minres_project(defl, np.zeros(op.n), b.copy())
    # span(AY) = span(Y) for exact eigenvectors, so the new residual is orthogonal to Y
    assert np.max(np.abs(Y.T @ r2)) < 1e-12 * np.linalg.norm(b)


def test_bicgstab_scalar_matrix_one_half_step():
    lam = 3.7
    b = gi.rhs(50, 5)
    res = krylov.bicgstab_cycle(lambda u: lam * u, np.zeros(50), b, 1e-12 * np.linalg.norm(b))
    assert res.converged and res.mvps == 1
    assert _rel(res.x, b / lam) < 1e-15


@pytest.mark.parametrize("kind,N,beta", [(CD2D, 15, (1.0,)), (CD3D, 7, (2.0, 1.0, 0.5))])
def test_bicgstab_brute_force(kind, N, beta):
    op = Operator(kind, N, beta)
    b = gi.rhs(op.n, 6)
    xs = _dense_solve(op, b)
    for ncyc, cap in ((1, None), (0, 20), (10, None)):
        res = krylov.bicgstab_proj(op.apply, b, np.zeros(op.n), None, rtol=1e-11,
                                   ncyc=ncyc, restart_mvps=cap, max_mvps=20000)
        assert res.converged
        assert _rel(res.x, xs) < 1e-8
        assert res.relres <= 1e-11


def test_bicgstab_cycle_recurrences():
    op = Operator(CD2D, 15, (1.0,))
    b = gi.rhs(op.n, 7)
    # half step only: s = r - alpha v is orthogonal to the shadow vector r_hat = r0
    res = krylov.bicgstab_cycle(op.apply, np.zeros(op.n), b, 0.0, max_mvps=1)
    assert abs(b @ res.r) < 1e-12 * np.linalg.norm(b) * np.linalg.norm(res.r)
    assert _rel(res.r, b - op.apply(res.x)) < 1e-12
    # full steps: the recursively updated residual stays equal to b - A x
    res = krylov.bicgstab_cycle(op.apply, np.zeros(op.n), b, 0.0, max_mvps=12)
    assert res.mvps == 12
    assert _rel(res.r, b - op.apply(res.x)) < 1e-10


def test_gmres_full_space_is_exact():
    op = Operator(CD2D, 5, (3.0,))
    b = gi.rhs(op.n, 8)
    res = krylov.gmres_cycle(op.apply, np.zeros(op.n), b, op.n, 0.0)
    assert _rel(res.x, _dense_solve(op, b)) < 1e-10
    assert all(res.history[i + 1] <= res.history[i] * (1 + 1e-12) for i in range(len(res.history) - 1))


def test_gmres_proj_brute_force():
    op = Operator(CD2D, 15, (1.0,))
    b = gi.rhs(op.n, 9)
    lam, W = np.linalg.eig(op.sparse().toarray())
    Y = W[:, np.argsort(lam.real)[:8]].real
    defl = krylov.make_deflation(op.apply, Y, "minres")
    res = krylov.gmres_proj(op.apply, b, np.zeros(op.n), defl, m=10, rtol=1e-11)
    assert res.converged and _rel(res.x, _dense_solve(op, b)) < 1e-8
    plain = krylov.gmres_proj(op.apply, b, np.zeros(op.n), None, m=10, rtol=1e-11)
    assert res.mvps < plain.mvps


def test_cycle_tolerance_schedule():
    rtol, ncyc, nr0 = 1e-8, 7, 3.0
    nr = nr0
    for icyc in range(1, ncyc + 1):
        rt = krylov.cycle_tolerance(rtol, nr0, nr, icyc, ncyc)
        # the second criterion: at least icyc/ncyc of the way in orders of magnitude
        assert rt * nr <= nr0 * rtol ** (icyc / ncyc) * (1 + 1e-12)
        nr = rt * nr
    assert abs(nr - rtol * nr0) < 1e-12 * rtol * nr0
    # a residual that jumped up during the projection: the second criterion is the binding one
    rt = krylov.cycle_tolerance(rtol, 1.0, 1e-2, 6, 20)
    assert abs(rt * 1e-2 - rtol ** (6 / 20)) < 1e-12


def test_harmonic_ritz_petrov_galerkin():
    op = Operator(CD2D, 15, (2.0,))
    m = 12
    V = np.zeros((op.n, m + 1))
    H = np.zeros((m + 1, m))
    b = gi.rhs(op.n, 10)
    V[:, 0] = b / np.linalg.norm(b)
    V, H = arnoldi_extend(op.apply, V, H, 0, m)
    theta, G = harmonic_ritz(H)
    AV = np.stack([op.apply(V[:, j]) for j in range(m)], axis=1)
    for i in range(m):
        y = V[:, :m] @ G[:, i]
        resid = AV @ G[:, i] - theta[i] * y
        assert np.linalg.norm(AV.T @ resid) < 1e-8 * np.linalg.norm(AV) * np.linalg.norm(y) * abs(theta[i])
    idx = select_k(theta, 4, True)
    er = eigen_residuals(H, theta, G, idx)
    for e, i in zip(er, idx):
        g = G[:, i] / np.linalg.norm(G[:, i])
        y = V[:, :m] @ g
        assert abs(e - np.linalg.norm(AV @ g - theta[i] * y)) < 1e-9 * abs(theta[i])


def test_gmresdr_single_cycle_is_gmres():
    op = Operator(CD2D, 15, (1.0,))
    b = gi.rhs(op.n, 11)
    gd = gmresdr(op.apply, b, 20, 5, max_cycles=1, rtol=0.0)
    ref = krylov.gmres_cycle(op.apply, np.zeros(op.n), b, 20, 0.0)
    assert _rel(gd.x, ref.x) < 1e-10


def test_gmresdr_ritz_values_converge_to_closed_form():
    N = 31
    op = Operator(CD2D, N, (1.0,))
    b = gi.rhs(op.n, 12)
    gd = gmresdr(op.apply, b, 30, 10, nev=6, rtolev=1e-9, rtol=1e-10, max_cycles=400)
    assert gd.converged
    exact = cd2d_eigenvalues(N, 1.0)[:6]
    th = np.sort(gd.theta.real)[:6]
    assert np.max(np.abs(th - exact) / exact) < 1e-8
    assert _rel(gd.x, _dense_solve(op, b)) < 1e-7
    # the returned basis is orthonormal and spans the converged eigenvectors
    Q = gd.Yc
    assert np.max(np.abs(Q.T @ Q - np.eye(Q.shape[1]))) < 1e-12
    lam, W = np.linalg.eig(op.sparse().toarray())
    w1 = W[:, np.argsort(lam.real)[0]].real
    assert np.linalg.norm(w1 - Q @ (Q.T @ w1)) < 1e-6


def test_gmresdr_complex_hermitian():
    L = 4
    op = Operator(U1_4D, L, links=gi.u1_links(L, 1), mass=0.05)
    b = gi.rhs(op.n, 13).astype(np.complex128)
    gd = gmresdr(op.apply, b, 30, 8, nev=4, rtolev=1e-8, rtol=1e-10, max_cycles=300,
                 dtype=np.complex128)
    assert gd.converged
    lam = np.linalg.eigvalsh(op.sparse().toarray())
    assert np.max(np.abs(np.sort(gd.theta.real)[:4] - lam[:4]) / lam[:4]) < 1e-7
    assert _rel(gd.x, np.linalg.solve(op.sparse().toarray(), b)) < 1e-7


@pytest.mark.parametrize("method", ["bicgstab", "gmres"])
@pytest.mark.parametrize("kind,N,beta", [(CD2D, 15, (1.0,)), (CD3D, 7, (2.0, 1.0, 0.5))])
def test_two_grid_brute_force(method, kind, N, beta):
    op = Operator(kind, N, beta)
    b = gi.rhs(op.n, 14)
    res = twogrid.two_grid_solve(op, b, m=12, k=4, rtolev=1e-6, method=method, rtol=1e-11,
                                 ncyc=10, restart_mvps=None, m3=8)
    assert res.solve.converged
    assert _rel(res.x, _dense_solve(op, b)) < 1e-8


def test_two_grid_lattice_brute_force():
    L = 8
    links = gi.u1_links(L, 2)
    op = Operator(U1_4D, L, links=links, mass=0.5)
    b = (gi.rhs(op.n, 15) + 0j)
    res = twogrid.two_grid_solve(op, b, m=20, k=8, rtolev=1e-4, rtol=1e-10, ncyc=10,
                                 restart_mvps=None)
    assert res.solve.converged
    xs = twogrid.exact_solution(op, b)
    assert _rel(res.x, xs) < 1e-7


def test_exact_solution_matches_dense():
    op = Operator(VARK2D, 9, (1.0,), gi.kappa_grf(9, 5))
    b = gi.rhs(op.n, 16)
    assert _rel(twogrid.exact_solution(op, b), _dense_solve(op, b)) < 1e-12


def test_adjoint_gradient_vs_finite_differences():
    N = 15
    kap = gi.kappa_grf(N, 3)
    op = Operator(VARK2D, N, (1.0,), kap)
    b = gi.rhs(op.n, 17)
    xstar = gi.random_dense(op.n, 18) * 1e-3
    _, grad, _, _ = adjoint.loss_and_gradient(op, b, xstar)
    nodes = gi.kappa_fd_nodes(N, 12, 0)
    fd = adjoint.finite_difference(op, b, xstar, nodes)
    assert np.max(np.abs(grad[nodes] - fd) / np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())) < 1e-5
    # a boundary node touching one interior face
    p = np.array([0 * (N + 2) + 5])
    fdb = adjoint.finite_difference(op, b, xstar, p)
    assert abs(grad[p][0] - fdb[0]) <= 1e-5 * max(abs(fdb[0]), 1e-3 * np.abs(fd).max())


@pytest.mark.parametrize("complex_", [False, True])
def test_harmonic_residual_identity(complex_):
    """The residual of every harmonic Ritz pair is a multiple of one vector: for an eigenpair
    (theta, g) of H_m + |h|^2 f e_m^T with H_m^H f = e_m, Hbar g - theta [g; 0] = g_m z with
    z = [-|h|^2 f; h].  The GPU restart kernel evaluates ||.|| this way; here the identity is
    checked against the explicit residual (oracle) on random and Arnoldi Hessenberg matrices."""
    m = 24
    H = gi.random_hessenberg(m, 3)
    if complex_:
        H = H + 1j * gi.random_hessenberg(m, 4)
    H = H + 3.0 * np.vstack([np.eye(m), np.zeros((1, m))])
    theta, G = harmonic_ritz(H)
    h = H[m, m - 1]
    f = np.linalg.solve(H[:m, :m].conj().T, np.eye(m)[:, -1])
    z = np.concatenate([-abs(h) ** 2 * f, [h]])
    idx = np.arange(m)
    explicit = eigen_residuals(H, theta, G, idx)
    for i in idx:
        g = G[:, i] / np.linalg.norm(G[:, i])
        gz = np.concatenate([g, [0.0]])
        r = H @ g - theta[i] * gz
        assert np.linalg.norm(r - g[-1] * z) <= 1e-10 * np.linalg.norm(H) * max(1.0, np.linalg.norm(z))
    assert np.allclose(explicit, np.abs(G[-1, :] / np.linalg.norm(G, axis=0)) * np.linalg.norm(z),
                       rtol=1e-8, atol=1e-12 * np.linalg.norm(H))


def test_finite_difference_equals_plain_subtraction_when_well_conditioned():
    """The oracle's central difference, formed from the solution change, equals the plain
    (L(kappa + h) - L(kappa - h)) / 2h of two separately solved losses where the plain form
    has digits to spare (a small grid and a small loss), and matches the adjoint gradient."""
    N = 11
    kap = gi.kappa_grf(N, 5)
    op = Operator(VARK2D, N, (1.0,), kap)
    b = gi.rhs(op.n, 21)
    x0 = adjoint.solve(op, b)
    xstar = x0 + 1e-2 * gi.random_dense(op.n, 22)           # a small loss, so subtraction keeps digits
    nodes = gi.kappa_fd_nodes(N, 6, 1)
    fd = adjoint.finite_difference(op, b, xstar, nodes, rel_step=1e-3)
    plain = []
    for p in nodes:
        dk = 1e-3 * kap[p]
        vals = []
        for sgn in (+1, -1):
            k2 = kap.copy()
            k2[p] += sgn * dk
            x = adjoint.solve(Operator(VARK2D, N, (1.0,), k2), b)
            vals.append(0.5 * float((x - xstar) @ (x - xstar)))
        plain.append((vals[0] - vals[1]) / (2 * dk))
    plain = np.array(plain)
    assert np.allclose(fd, plain, rtol=1e-6, atol=1e-9 * np.abs(plain).max())
    _, grad, _, _ = adjoint.loss_and_gradient(op, b, xstar)
    assert np.allclose(grad[nodes], fd, rtol=1e-5, atol=1e-8 * np.abs(fd).max())


def _hessenberg_with_spectrum(blocks, seed):
    """A real upper Hessenberg matrix orthogonally similar to the block-diagonal matrix
    of the given 1x1 / 2x2 blocks (its eigenvalues are those of the blocks), and the
    orthogonal factor Q with M = Q B Q^T."""
    import scipy.linalg as sla
    n = sum(len(b) for b in blocks)
    B = np.zeros((n, n))
    i = 0
    for b in blocks:
        b = np.atleast_2d(np.asarray(b, dtype=float))
        B[i:i + len(b), i:i + len(b)] = b
        i += len(b)
    Q0 = np.linalg.qr(gi.random_dense((n, n), seed))[0]
    Hm, Qh = sla.hessenberg(Q0 @ B @ Q0.T, calc_q=True)    # Q0 B Q0^T = Qh Hm Qh^T
    return Hm, (Qh.T @ Q0)


@pytest.mark.parametrize("k,kk_expected", [(1, 1), (2, 2), (3, 4), (4, 4), (5, 5)])
def test_select_k_conjugate_pair_rule(k, kk_expected):
    """Section 2.1 keeps k harmonic Ritz vectors; a real basis cannot hold one member of a
    complex-conjugate pair without its partner, so when the k-th value (order |theta|,
    Re, Im >= 0 first) is the Im > 0 member, k + 1 are kept.  With h_{m+1,m} = 0 the
    harmonic Ritz values are the eigenvalues of H_m, fixed here by construction:
    1, 2, 3 +- i (|.| = sqrt 10), 5, 7."""
    blocks = [[1.0], [2.0], [[3.0, 1.0], [-1.0, 3.0]], [5.0], [7.0]]
    Hm, Q = _hessenberg_with_spectrum(blocks, 41)
    m = Hm.shape[0]
    Hbar = np.vstack([Hm, np.zeros((1, m))])
    theta, G = harmonic_ritz(Hbar)
    idx = select_k(theta, k, True)
    assert len(idx) == kk_expected
    want = np.array([1.0, 2.0, 3.0 + 1.0j, 3.0 - 1.0j, 5.0, 7.0])[:kk_expected]
    assert np.allclose(theta[idx], want, atol=1e-12)
    # the real basis spans exactly the invariant subspace of the kept values (both partners):
    # B's invariant subspace of its first kk coordinates, mapped by Q
    from oracle.gmresdr import real_span_basis
    Bk = np.linalg.qr(real_span_basis(G, theta, idx, True))[0]
    assert Bk.shape[1] == kk_expected
    exact = Q[:, :kk_expected]                  # orthonormal, spans the same subspace
    s = np.linalg.svd(exact.T @ Bk, compute_uv=False)
    assert np.min(s) > 1 - 1e-10                  # cosines of the principal angles


def test_select_k_complex_problem_keeps_k():
    """Complex arithmetic needs no partner: exactly k are kept even when the k-th value
    has a conjugate partner in the spectrum."""
    blocks = [[1.0], [[3.0, 1.0], [-1.0, 3.0]], [5.0]]
    Hm, _ = _hessenberg_with_spectrum(blocks, 42)
    Hbar = np.vstack([Hm, np.zeros((1, Hm.shape[0]))]).astype(np.complex128)
    theta, _ = harmonic_ritz(Hbar)
    assert len(select_k(theta, 2, False)) == 2


def test_bicgstab_proj_continues_past_ncyc():
    """Reading of Section 4.1 step 3: when the ncyc scheduled cycles end above rtol (here
    each is capped at 10 products), the solve goes on with cycles aiming at rtol, and
    still reaches the dense-LU solution."""
    op = Operator(CD2D, 15, (1.0,))
    b = gi.rhs(op.n, 7)
    res = krylov.bicgstab_proj(op.apply, b, np.zeros(op.n), None, rtol=1e-11, ncyc=2,
                               restart_mvps=10, max_mvps=20000)
    assert res.converged and res.cycles > 2
    assert _rel(res.x, _dense_solve(op, b)) < 1e-8
    for icyc, relres, rt, _ in res.history[2:]:
        assert abs(rt * relres - 1e-11) <= 1e-11 * 1e-12


def test_idr1_is_bicgstab():
    """IDR(1) with the shadow vector r0 / ||r0|| and omega taken as the plain minimiser
    (kappa = 0) is BiCGStab (Sonneveld and van Gijzen's equivalence): the residual norms
    after every product agree with the textbook BiCGStab cycle's half and full steps."""
    op = Operator(CD2D, 15, (5.0,))
    b = gi.rhs(op.n, 3)
    P = (b / np.linalg.norm(b))[:, None]
    ri = krylov.idr_cycle(op.apply, np.zeros(op.n), b, P, 0.0, max_mvps=24, kappa=0.0)
    rb = krylov.bicgstab_cycle(op.apply, np.zeros(op.n), b, 0.0, max_mvps=24)
    assert len(ri.history) == len(rb.history) == 24
    assert np.allclose(ri.history, rb.history, rtol=1e-9, atol=0)
    assert _rel(ri.x, rb.x) < 1e-9


def test_idr_finite_termination():
    """In exact arithmetic IDR(s) solves an n x n system within n + n/s products; on a
    well-conditioned dense nonsymmetric 12 x 12 system with s = 4 it reaches rounding level
    within 15."""
    n, s = 12, 4
    A = gi.random_dense((n, n), 21) + 4 * np.eye(n)
    b = gi.random_dense(n, 22)
    P = krylov.shadow_space(gi.random_dense((n, s), 23))
    res = krylov.idr_cycle(lambda v: A @ v, np.zeros(n), b, P, 1e-12 * np.linalg.norm(b), max_mvps=40)
    assert res.converged and res.mvps <= n + n // s
    assert _rel(res.x, np.linalg.solve(A, b)) < 1e-10


def test_idr_scalar_matrix_one_product():
    """A = lambda I: the first IDR(s) step already gives the exact solution (one product)."""
    n = 50
    b = gi.random_dense(n, 24)
    P = krylov.shadow_space(gi.random_dense((n, 4), 25))
    res = krylov.idr_cycle(lambda v: 3.5 * v, np.zeros(n), b, P, 1e-13 * np.linalg.norm(b))
    assert res.mvps == 1 and _rel(res.x, b / 3.5) < 1e-14


def test_shadow_space_unique():
    """The positive-diagonal QR convention fixes the orthonormal shadow space: it equals
    Gram-Schmidt of the random columns in order, and P^H P = I."""
    R0 = gi.random_dense((40, 4), 26)
    P = krylov.shadow_space(R0)
    assert np.allclose(P.T @ P, np.eye(4), atol=1e-14)
    Q = np.zeros_like(R0)
    for j in range(4):
        w = R0[:, j] - Q[:, :j] @ (Q[:, :j].T @ R0[:, j])
        Q[:, j] = w / np.linalg.norm(w)
    assert np.allclose(P, Q, atol=1e-13)


@pytest.mark.parametrize("kind,N,beta", [(CD2D, 15, (1.0,)), (CD3D, 7, (2.0, 1.0, 0.5))])
def test_idr_proj_brute_force(kind, N, beta):
    op = Operator(kind, N, beta)
    b = gi.rhs(op.n, 27)
    xs = _dense_solve(op, b)
    P = krylov.shadow_space(gi.random_dense((op.n, 4), 28))
    Y = gi.random_dense((op.n, 6), 29)
    defl = krylov.make_deflation(op.apply, Y, "minres")
    for ncyc, cap in ((10, None), (0, 25), (3, 9)):
        res = krylov.idr_proj(op.apply, b, np.zeros(op.n), defl, P, rtol=1e-11, ncyc=ncyc,
                              restart_mvps=cap, max_mvps=20000)
        assert res.converged and _rel(res.x, xs) < 1e-8


def test_arnoldi_e_symmetric_monotone_and_interlacing():
    """Every Arnoldi-E cycle works in a subspace containing the previous span(Y), so for a
    symmetric matrix (cd2d with beta = 0) the j-th smallest kept Ritz value can only go down
    (Courant-Fischer) and never below the j-th eigenvalue (Cauchy interlacing); the values
    approach the closed-form eigenvalues."""
    from oracle.gmresdr import arnoldi_e
    N, k = 31, 8
    op = Operator(CD2D, N, (0.0,))
    lam = cd2d_eigenvalues(N, 0.0)
    Y = gi.random_dense((op.n, k), 31)
    prev = None
    for c in range(0, 7):
        _, th, _, _, _ = arnoldi_e(op.apply, Y, 30, c, 4)
        t = np.sort(th.real)[:k]
        assert np.all(np.abs(th.imag) == 0)
        assert np.all(t >= lam[:k] - 1e-9 * lam[-1])
        if prev is not None:
            assert np.all(t <= prev + 1e-9 * lam[-1])
        prev = t
    assert abs(prev[0] - lam[0]) <= 1e-6 * lam[0]


def test_arnoldi_e_keeps_an_invariant_subspace():
    """Exact eigenvectors (closed form for beta = 0: products of sines) give Ritz values
    equal to their eigenvalues with zero residual, cycle after cycle."""
    from oracle.gmresdr import arnoldi_e
    N = 31
    op = Operator(CD2D, N, (0.0,))
    h = 1.0 / (N + 1)
    t = np.arange(1, N + 1) * h
    modes = [(1, 1), (1, 2), (2, 1), (2, 2), (1, 3), (3, 1)]
    Y = np.stack([np.outer(np.sin(q * np.pi * t), np.sin(p * np.pi * t)).reshape(-1) for p, q in modes], axis=1)
    exact = np.sort([(4 - 2 * np.cos(p * np.pi * h) - 2 * np.cos(q * np.pi * h)) / h**2 for p, q in modes])
    _, th, eres, _, _ = arnoldi_e(op.apply, Y, 20, 2, 2)
    assert np.allclose(np.sort(th.real), exact, rtol=1e-10)
    assert np.max(eres) <= 1e-9 * exact[-1]
