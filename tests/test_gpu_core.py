"""GPU parity of the building blocks against the oracle (through the C ABI).

Tolerances (the method's own numbers where it gives them):
  * per operator application: relative difference <= 1e-13 in float64 (norm-wise and
    max-abs relative to max |y|); float32 applications <= 1e-6;
  * grid maps: bilinear / trilinear prolongation bit-exact (same summation order);
    lattice transfer and restriction <= 1e-15 relative (complex products may round
    differently);
  * projection: the oracle's Householder-QR MinRes / Galerkin projection to <= 1e-11
    relative (CholQR2 and Householder differ by rounding amplified by cond(A Y)); the
    invariant (A Y)^T r_new = 0 to 1e-12 ||A Y|| ||r||; ||Q^T Q - I|| <= 1e-13;
  * harmonic Ritz kernel: values to 1e-10 relative, the kept span to 1e-8 (sine of the
    largest principal angle) against numpy eig on the same matrix.
"""
import numpy as np
import pytest

import tg_inputs as gi
from oracle import krylov, transfer
from oracle.gmresdr import eigen_residuals, harmonic_ritz as o_hritz, order_ritz, real_span_basis, select_k
from oracle.operators import CD2D, CD3D, U1_4D, VARK2D, Operator as OOp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_03070_gb300 import build
    build.build()
    from paper_2005_03070_gb300 import tg as mod
    mod.load()
    return mod


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def make_pair(tg, kind, N, beta=(1.0,), seed=0, mass=0.1):
    if kind == "vark2d":
        kap = gi.kappa_grf(N, seed)
        return tg.Operator(kind, N, beta, kappa=cu(kap)), OOp(VARK2D, N, beta, kap)
    if kind == "u1_4d":
        links = gi.u1_links(N, seed)
        return (tg.Operator(kind, N, links=cu(links), mass=mass),
                OOp(U1_4D, N, links=links, mass=mass))
    k = {"cd2d": CD2D, "cd3d": CD3D}[kind]
    return tg.Operator(kind, N, beta), OOp(k, N, beta)


CASES = [("cd2d", 127, (1.0,)), ("cd2d", 33, (-7.0,)), ("cd3d", 31, (2.0, 1.0, 0.5)),
         ("vark2d", 63, (1.0,)), ("u1_4d", 8, None)]


@pytest.mark.parametrize("kind,N,beta", CASES)
@pytest.mark.parametrize("transpose", [False, True])
def test_per_matvec_parity(tg, kind, N, beta, transpose):
    top, oop = make_pair(tg, kind, N, beta or (0.0,))
    rng = np.random.default_rng(3)
    u = rng.standard_normal(oop.n) + (1j * rng.standard_normal(oop.n) if oop.kind == U1_4D else 0)
    y = host(top.apply(cu(u), transpose=transpose))
    if transpose:
        ref = (oop.sparse().conj().T @ u)
    else:
        ref = oop.apply(u)
    assert rel(y, ref) <= 1e-13
    assert np.max(np.abs(y - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("kind,N,beta", [c for c in CASES if c[0] != "u1_4d"])
def test_per_matvec_float32(tg, kind, N, beta):
    top, oop = make_pair(tg, kind, N, beta)
    u = np.random.default_rng(4).standard_normal(oop.n)
    y = host(top.apply(cu(u.astype(np.float32)), precision=tg.TG_F32_IR)).astype(np.float64)
    assert rel(y, oop.apply(u)) <= 1e-6


@pytest.mark.parametrize("kind,N,beta", [c for c in CASES if c[0] != "u1_4d"])
def test_coarse_operator_parity(tg, kind, N, beta):
    from oracle.operators import coarse_operator
    top, oop = make_pair(tg, kind, N, beta)
    opc = coarse_operator(oop)
    u = np.random.default_rng(5).standard_normal(opc.n)
    y = host(top.apply(cu(u), level=tg.TG_COARSE))
    assert rel(y, opc.apply(u)) <= 1e-13


def test_lattice_coarse_galerkin_parity(tg):
    top, oop = make_pair(tg, "u1_4d", 8)
    Ac, P, *_ = transfer.lattice_coarse_stencil(oop)
    rng = np.random.default_rng(6)
    v = rng.standard_normal(Ac.shape[0]) + 1j * rng.standard_normal(Ac.shape[0])
    y = host(top.apply(cu(v), level=tg.TG_COARSE))
    assert rel(y, Ac @ v) <= 1e-13
    f = host(top.prolong(cu(v)))
    assert rel(f, P @ v) <= 1e-15
    w = rng.standard_normal(P.shape[0]) + 1j * rng.standard_normal(P.shape[0])
    assert rel(host(top.restrict(cu(w))), P.conj().T @ w) <= 1e-14


@pytest.mark.parametrize("kind,N", [("cd2d", 127), ("cd2d", 9), ("cd3d", 31), ("cd3d", 7)])
def test_prolongation_bit_exact(tg, kind, N):
    top, oop = make_pair(tg, kind, N, (1.0,) if kind == "cd2d" else (2.0, 1.0, 0.5))
    Nc = (N - 1) // 2
    dim = 2 if kind == "cd2d" else 3
    rng = np.random.default_rng(7)
    uc = rng.standard_normal((3, Nc ** dim))
    f = host(top.prolong(cu(uc.reshape(-1)))).reshape(3, -1)
    for c in range(3):
        ref = transfer.prolong2d(uc[c], Nc) if dim == 2 else transfer.prolong3d(uc[c], Nc)
        assert np.array_equal(f[c], ref)
    uf = rng.standard_normal(N ** dim)
    r = host(top.restrict(cu(uf)))
    assert rel(r, transfer.restrict(uf, N, dim)) <= 1e-14


@pytest.mark.parametrize("kind,N", [("cd2d", 127), ("cd2d", 7), ("cd2d", 3), ("cd3d", 31), ("cd3d", 7), ("cd3d", 3)])
def test_cubic_prolongation_bit_exact(tg, kind, N):
    """The cubic interpolation (stand-in for the paper's splines) against the oracle, bit for
    bit: same fixed summation order; N = 3 (Nc = 1) has every stencil folded at the boundary."""
    dim = 2 if kind == "cd2d" else 3
    top = tg.Operator(kind, N, (1.0,) if dim == 2 else (2.0, 1.0, 0.5), interp="cubic")
    Nc = (N - 1) // 2
    rng = np.random.default_rng(17)
    uc = rng.standard_normal((3, Nc ** dim))
    f = host(top.prolong(cu(uc.reshape(-1)))).reshape(3, -1)
    for c in range(3):
        ref = transfer.prolong2d_cubic(uc[c], Nc) if dim == 2 else transfer.prolong3d_cubic(uc[c], Nc)
        assert np.array_equal(f[c], ref)
    # the restriction is unchanged (full weighting)
    uf = rng.standard_normal(N ** dim)
    assert rel(host(top.restrict(cu(uf))), transfer.restrict(uf, N, dim)) <= 1e-14


def test_interp_setter_rejects_the_lattice_and_unknown_values(tg):
    top, _ = make_pair(tg, "u1_4d", 8)
    lib = tg.load()
    assert lib.tg_op_set_interp(top.handle, 1) == tg.TG_BAD_ARG
    g = tg.Operator("cd2d", 15, (1.0,))
    assert lib.tg_op_set_interp(g.handle, 7) == tg.TG_BAD_ARG
    assert lib.tg_op_set_interp(g.handle, 1) == 0


@pytest.mark.parametrize("proj", ["minres", "galerkin"])
@pytest.mark.parametrize("kind,N,beta", [("cd2d", 63, (1.0,)), ("cd3d", 15, (2.0, 1.0, 0.5))])
def test_projection_parity(tg, proj, kind, N, beta):
    top, oop = make_pair(tg, kind, N, beta)
    k = 12
    Y = gi.random_dense((oop.n, k), 8)
    defl = top.defl_from_basis(cu(Y.T.copy().reshape(-1)), k, proj=proj)
    odefl = krylov.make_deflation(oop.apply, Y, proj)
    b = gi.rhs(oop.n, 9)
    x0 = gi.random_dense(oop.n, 10)
    r0 = b - oop.apply(x0)
    xo, ro = krylov.project(odefl, x0, r0)
    xt, rt = cu(x0), cu(r0)
    defl.project(xt, rt)
    xg, rg = host(xt), host(rt)
    assert rel(xg, xo) <= 1e-11
    assert rel(rg, ro) <= 1e-11
    AY = odefl.AY
    W = AY if proj == "minres" else np.linalg.qr(Y)[0]
    assert np.max(np.abs(W.T @ rg)) <= 1e-12 * np.linalg.norm(W) * np.linalg.norm(r0)
    Q = host(defl.copy(1)).T
    assert np.max(np.abs(Q.T @ Q - np.eye(k))) <= 1e-13
    assert np.max(np.abs(host(defl.copy(2)).T - AY)) <= 1e-13 * np.max(np.abs(AY))


@pytest.mark.parametrize("proj", ["minres", "galerkin"])
def test_projection_parity_complex(tg, proj):
    """Complex projection (lattice operator, 6^4 sites): the same bars with conjugate
    transposes."""
    top, oop = make_pair(tg, "u1_4d", 6, None, seed=3)
    k = 10
    Y = gi.random_dense((oop.n, k), 8) + 1j * gi.random_dense((oop.n, k), 18)
    defl = top.defl_from_basis(cu(Y.T.copy().reshape(-1)), k, proj=proj)
    odefl = krylov.make_deflation(oop.apply, Y, proj)
    b = gi.rhs(oop.n, 9) + 1j * gi.rhs(oop.n, 19)
    x0 = gi.random_dense(oop.n, 10) + 1j * gi.random_dense(oop.n, 20)
    r0 = b - oop.apply(x0)
    xo, ro = krylov.project(odefl, x0, r0)
    xt, rt = cu(x0), cu(r0)
    defl.project(xt, rt)
    xg, rg = host(xt), host(rt)
    assert rel(xg, xo) <= 1e-11
    assert rel(rg, ro) <= 1e-11
    AY = odefl.AY
    W = AY if proj == "minres" else np.linalg.qr(Y)[0]
    assert np.max(np.abs(W.conj().T @ rg)) <= 1e-12 * np.linalg.norm(W) * np.linalg.norm(r0)
    Q = host(defl.copy(1)).T
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(k))) <= 1e-13


def _span_gap(A, B):
    """sin of the largest principal angle between span(A) and span(B) (columns)."""
    Qa = np.linalg.qr(A)[0]
    Qb = np.linalg.qr(B)[0]
    return np.linalg.norm(Qb - Qa @ (Qa.conj().T @ Qb), 2)


def _arnoldi_hessenberg(m, seed):
    """Hbar of m Arnoldi steps on a convection-diffusion operator (what GMRES-DR feeds the
    kernel: eigenvectors far better conditioned than those of a random matrix)."""
    from oracle.gmresdr import arnoldi_extend
    op = OOp(CD2D, 63, (3.0,))
    V = np.zeros((op.n, m + 1))
    H = np.zeros((m + 1, m))
    b = gi.rhs(op.n, seed)
    V[:, 0] = b / np.linalg.norm(b)
    return arnoldi_extend(op.apply, V, H, 0, m)[1]


@pytest.mark.parametrize("m,k,seed,src", [(12, 4, 0, "rand"), (30, 15, 1, "rand"), (60, 30, 2, "rand"),
                                         (80, 40, 3, "arnoldi"), (128, 60, 4, "arnoldi")])
def test_harmonic_ritz_kernel_real(tg, m, k, seed, src):
    if src == "rand":
        H = gi.random_hessenberg(m, seed)
        H[:, :] += 3.0 * np.vstack([np.eye(m), np.zeros((1, m))])     # keep H_m well conditioned
    else:
        H = _arnoldi_hessenberg(m, seed)
    th, basis, eres = tg.harmonic_ritz(cu(H.T.copy()), m, k)
    th, basis, eres = host(th), host(basis).T, host(eres)
    theta, G = o_hritz(H)
    idx = order_ritz(theta)
    assert np.max(np.abs(th - theta[idx]) / np.abs(theta[idx])) <= 1e-10
    sel = select_k(theta, k, True)
    assert basis.shape[1] == len(sel)
    ref = real_span_basis(G, theta, sel, True)
    assert _span_gap(ref, basis) <= 1e-8
    assert np.max(np.abs(basis.T @ basis - np.eye(len(sel)))) <= 1e-12
    # eigen-residuals ||Hbar g - theta [g; 0]|| (the oracle forms them explicitly)
    ref_res = eigen_residuals(H, theta, G, idx[:len(sel)])
    assert np.allclose(eres, ref_res, rtol=1e-6, atol=1e-10 * np.linalg.norm(H))


@pytest.mark.parametrize("m,k,seed", [(20, 6, 5), (40, 20, 6)])
def test_harmonic_ritz_kernel_complex(tg, m, k, seed):
    H = gi.random_hessenberg(m, seed) + 1j * gi.random_hessenberg(m, seed + 100)
    H += 3.0 * np.vstack([np.eye(m), np.zeros((1, m))])
    th, basis, eres = tg.harmonic_ritz(cu(H.T.copy()), m, k, complex_=True)
    th, basis = host(th), host(basis).T
    theta, G = o_hritz(H)
    idx = order_ritz(theta)
    assert np.max(np.abs(th - theta[idx]) / np.abs(theta[idx])) <= 1e-10
    sel = select_k(theta, k, False)
    assert _span_gap(G[:, sel], basis) <= 1e-8
    ref_res = eigen_residuals(H, theta, G, idx[:len(sel)])
    assert np.allclose(host(eres), ref_res, rtol=1e-6, atol=1e-10 * np.linalg.norm(H))


@pytest.mark.parametrize("kind,N,beta", [("cd2d", 63, (1.0,)), ("u1_4d", 8, None)])
def test_bicgstab_partial_cycle_parity(tg, kind, N, beta):
    top, oop = make_pair(tg, kind, N, beta or (0.0,), mass=0.5)
    b = gi.rhs(oop.n, 11).astype(oop.dtype)
    x0 = np.zeros(oop.n, dtype=oop.dtype)
    for mv in (1, 2, 7, 12):
        ref = krylov.bicgstab_proj(oop.apply, b, x0, None, rtol=1e-14, ncyc=0, restart_mvps=mv, max_mvps=mv)
        xt = cu(x0.copy())
        st, stats = top.solve(cu(b), xt, rtol=1e-14, ncyc=0, restart_mvps=mv, max_mvps=mv)
        assert stats[0]["mvps"] == ref.mvps == mv
        assert rel(host(xt), ref.x) <= 1e-11
