"""GPU parity of the rows beyond the core path (through the C ABI): the paper's Example 1
operator -exp(5xy) Lap u + 40 u_x + 40 u_y, the Helmholtz operator of Example 4 as a
reaction shift, IDR(s)-Proj (Section 4.1), and GMRES-DR / Gram / projection at the paper's
large sizes (m up to 200, k up to 150).

Bars: per operator application <= 1e-13 relative (float64) and <= 1e-6 (float32); an IDR
cycle of a given number of products gives the oracle's iterate to 1e-10 (the kernels
biorthogonalise in the classical form, the oracle one column at a time: equal in exact
arithmetic); end-to-end solves reach rtol = 1e-10 by the oracle's operator and the
sparse-LU solution to 1e-6; harmonic Ritz values at m = 150 and 200 agree with numpy's eig
to 1e-9 relative and the kept spans to 1e-6.
"""
import numpy as np
import pytest

import tg_inputs as gi
from oracle import krylov, transfer, twogrid
from oracle.gmresdr import gmresdr, harmonic_ritz as o_hritz, select_k, real_span_basis
from oracle.operators import CD2D, EXP2D, U1_4D, Operator as OOp, coarse_operator

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EX1 = (40.0, 40.0, 5.0)


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


def _pairs(tg, N):
    return {"exp2d": (tg.Operator("exp2d", N, EX1), OOp(EXP2D, N, EX1)),
            "helmholtz": (tg.Operator("cd2d", N, (0.0,), mass=-1e4), OOp(CD2D, N, (0.0,), mass=-1e4))}


@pytest.mark.parametrize("name", ["exp2d", "helmholtz"])
def test_new_operators_apply(tg, name):
    top, oop = _pairs(tg, 127)[name]
    opc = coarse_operator(oop)
    for level, o in ((tg.TG_FINE, oop), (tg.TG_COARSE, opc)):
        u = gi.rhs(o.n, 41)
        for tr in (False, True):
            ref = (o.transposed() if tr else o).apply(u)
            y = host(top.apply(cu(u), level=level, transpose=tr))
            assert rel(y, ref) <= 1e-13, (level, tr)
            assert np.max(np.abs(y - ref)) <= 1e-13 * np.max(np.abs(ref))
        y32 = host(top.apply(cu(u.astype(np.float32)), level=level, precision=tg.TG_F32_IR)).astype(np.float64)
        assert rel(y32, o.apply(u)) <= 1e-6


def _two_grid(tg, top, b, m, k, method="bicgstab", **kw):
    bt = cu(b)
    xc, defl, cst, _ = top.coarse_gmresdr(bt, m, k, rtolev=1e-3, rtol=1e-8, max_cycles=300)
    x = top.prolong(xc)
    if method == "idr":
        P = cu(gi.random_dense((4, top.n), 42))
        status, st = top.solve_idr(bt, x, P, defl, rtol=1e-10, ncyc=kw.get("ncyc", 20))
    else:
        status, st = top.solve(bt, x, defl, method=method, rtol=1e-10, ncyc=kw.get("ncyc", 20), restart_mvps=0,
                               m3=kw.get("m3", 30))
    return host(x), status, st[0]


@pytest.mark.parametrize("method", ["bicgstab", "gmres", "idr"])
def test_example1_two_grid(tg, method):
    top, oop = _pairs(tg, 127)["exp2d"]
    b = gi.rhs(oop.n, 43)
    xs = twogrid.exact_solution(oop, b)
    x, status, st = _two_grid(tg, top, b, 40, 20, method)
    assert status == tg.TG_OK, st
    assert np.linalg.norm(b - oop.apply(x)) / np.linalg.norm(b) <= 1e-10
    assert rel(x, xs) <= 1e-6


@pytest.mark.parametrize("case", ["exp2d", "helmholtz"])
def test_idr_float32_refinement_two_grid(tg, case):
    """IDR(4)-Proj in the float32 + refinement form: float32 IDR cycles on the correction
    equation (float32 shadow space and projection) with float64 refinement, on Example 1's
    operator (127^2) and on the indefinite Helmholtz case (63^2, -Lap u - 30^2 u, cubic
    prolongation).  The solution reaches rtol = 1e-10 (recomputed by the oracle's operator)
    and the direct solution to 1e-6."""
    if case == "exp2d":
        top, oop = _pairs(tg, 127)["exp2d"]
        m, k, ncyc = 40, 20, 20
    else:
        top = tg.Operator("cd2d", 63, (0.0,), mass=-900.0, interp="cubic")
        oop = OOp(CD2D, 63, (0.0,), mass=-900.0)
        m, k, ncyc = 40, 20, 10
    b = gi.rhs(oop.n, 46)
    xs = twogrid.exact_solution(oop, b)
    bt = cu(b)
    xc, defl, _, _ = top.coarse_gmresdr(bt, m, k, rtolev=1e-3, rtol=1e-8, max_cycles=300, precision="f32_ir")
    x = top.prolong(xc)
    P = cu(gi.random_dense((4, top.n), 42))
    status, st = top.solve_idr(bt, x, P, defl, rtol=1e-10, ncyc=ncyc, precision="f32_ir")
    assert status == tg.TG_OK, st
    xh = host(x)
    assert np.linalg.norm(b - oop.apply(xh)) / np.linalg.norm(b) <= 1e-10
    assert rel(xh, xs) <= 1e-6


@pytest.mark.parametrize("interp", ["linear", "cubic"])
@pytest.mark.parametrize("method", ["gmres", "idr"])
def test_helmholtz_two_grid(tg, method, interp):
    """-Lap u - 30^2 u on 63^2 (several negative eigenvalues): the indefinite case, with the
    moved vectors interpolated bilinearly and by the cubic stand-in for the paper's splines."""
    top = tg.Operator("cd2d", 63, (0.0,), mass=-900.0, interp=interp)
    oop = OOp(CD2D, 63, (0.0,), mass=-900.0)
    b = gi.rhs(oop.n, 44)
    xs = twogrid.exact_solution(oop, b)
    x, status, st = _two_grid(tg, top, b, 40, 20, method, ncyc=10, m3=40)
    assert status == tg.TG_OK, st
    assert rel(x, xs) <= 1e-6


@pytest.mark.parametrize("kind,N,s", [("cd2d", 63, 4), ("cd2d", 63, 1), ("cd2d", 63, 8), ("u1_4d", 6, 4)])
def test_idr_partial_cycle_parity(tg, kind, N, s):
    if kind == "u1_4d":
        links = gi.u1_links(N, 3)
        top = tg.Operator(kind, N, links=cu(links), mass=0.5)
        oop = OOp(U1_4D, N, links=links, mass=0.5)
        b = (gi.rhs(oop.n, 45) + 1j * gi.rhs(oop.n, 46)).astype(np.complex128)
        Praw = gi.random_dense((oop.n, s), 47) + 1j * gi.random_dense((oop.n, s), 48)
    else:
        top, oop = tg.Operator(kind, N, (3.0,)), OOp(CD2D, N, (3.0,))
        b = gi.rhs(oop.n, 45)
        Praw = gi.random_dense((oop.n, s), 47)
    P = krylov.shadow_space(Praw)
    x0 = np.zeros(oop.n, dtype=oop.dtype)
    for mv in sorted({1, 2, s, s + 1, s + 2, 12}):
        ref = krylov.idr_proj(oop.apply, b, x0, None, P, rtol=1e-14, ncyc=0, restart_mvps=mv, max_mvps=mv)
        xt = cu(x0.copy())
        st, stats = top.solve_idr(cu(b), xt, cu(Praw.T.copy()), None, rtol=1e-14, ncyc=0, restart_mvps=mv,
                                  max_mvps=mv)
        assert stats[0]["mvps"] == ref.mvps == mv
        assert rel(host(xt), ref.x) <= 1e-10, mv


def test_idr1_matches_bicgstab_on_gpu(tg):
    """IDR(1) with P = r0 and no angle safeguard is BiCGStab: the two GPU paths give the
    same iterate after 12 products."""
    top = tg.Operator("cd2d", 63, (3.0,))
    b = gi.rhs(63 * 63, 49)
    x1 = cu(np.zeros(b.size))
    x2 = cu(np.zeros(b.size))
    top.solve_idr(cu(b), x1, cu(b[None, :].copy()), None, rtol=1e-14, ncyc=0, restart_mvps=12, max_mvps=12,
                  kappa=0.0)
    top.solve(cu(b), x2, None, rtol=1e-14, ncyc=0, restart_mvps=12, max_mvps=12)
    assert rel(host(x1), host(x2)) <= 1e-10


def _arnoldi_hbar(m, complex_, seed):
    """Hbar of m Arnoldi steps (what GMRES-DR hands the restart kernel): Example 1's operator
    on 63^2, or the 6^4 U(1) lattice in complex arithmetic."""
    from oracle.gmresdr import arnoldi_extend
    if complex_:
        op = OOp(U1_4D, 6, links=gi.u1_links(6, seed), mass=0.5)
        b = (gi.rhs(op.n, seed) + 1j * gi.rhs(op.n, seed + 1)).astype(np.complex128)
    else:
        op = OOp(EXP2D, 63, EX1)
        b = gi.rhs(op.n, seed)
    V = np.zeros((op.n, m + 1), dtype=op.dtype)
    H = np.zeros((m + 1, m), dtype=op.dtype)
    V[:, 0] = b / np.linalg.norm(b)
    return arnoldi_extend(op.apply, V, H, 0, m)[1]


@pytest.mark.parametrize("m,k,complex_", [(150, 100, False), (200, 150, False), (150, 100, True)])
def test_harmonic_ritz_large_m(tg, m, k, complex_):
    from oracle.gmresdr import order_ritz
    H = _arnoldi_hbar(m, complex_, 50 + m)
    theta_o, G = o_hritz(H)
    th, basis, eres = tg.harmonic_ritz(cu(H.T.copy()), m, k, complex_=complex_)
    th = host(th)
    idx = order_ritz(theta_o)
    assert np.max(np.abs(th - theta_o[idx])) <= 1e-9 * np.max(np.abs(theta_o))
    sel = select_k(theta_o, k, not complex_)
    assert basis.shape[0] == len(sel)
    Bo = np.linalg.qr(real_span_basis(G, theta_o, sel, not complex_))[0]
    Bg = np.linalg.qr(host(basis).T)[0]
    c = np.clip(np.linalg.svd(Bo.conj().T @ Bg, compute_uv=False), 0, 1)
    assert np.max(np.sqrt(1 - c ** 2)) <= 1e-6


def test_gmresdr_cycle_m150_example1_coarse(tg):
    """One GMRES-DR(150,100) cycle (= GMRES(150)) on Example 1's 63^2 coarse grid."""
    top, oop = _pairs(tg, 127)["exp2d"]
    opc = coarse_operator(oop)
    b = gi.rhs(oop.n, 51)
    ref = gmresdr(opc.apply, transfer.restrict(b, 127, 2), 150, 100, rtolev=1e-12, rtol=1e-14, max_cycles=1)
    xc, _, st, _ = top.coarse_gmresdr(cu(b), 150, 100, rtolev=1e-12, rtol=1e-14, max_cycles=1, want_defl=False)
    assert rel(host(xc), ref.x) <= 1e-9


def test_projection_k150(tg):
    """A 150-vector deflation basis: CholQR2's Q is orthonormal and the MinRes projection
    matches the oracle's Householder-QR projection."""
    N = 127
    top, oop = tg.Operator("cd2d", N, (1.0,)), OOp(CD2D, N, (1.0,))
    Y = gi.random_dense((oop.n, 150), 52)
    defl = top.defl_from_basis(cu(Y.T.copy()), 150)
    Q = host(defl.copy(1)).T
    assert np.max(np.abs(Q.T @ Q - np.eye(150))) <= 1e-12
    r = gi.rhs(oop.n, 53)
    x = np.zeros(oop.n)
    xr, rr = krylov.minres_project(krylov.make_deflation(oop.apply, Y), x, r)
    xt, rt = cu(x), cu(r)
    defl.project(xt, rt)
    assert rel(host(rt), rr) <= 1e-9
    assert rel(host(xt), xr) <= 1e-8


@pytest.mark.parametrize("cycles", [0, 1, 3])
def test_arnoldi_e_matches_oracle(tg, cycles):
    """Arnoldi-E(24, 8) on Example 1's operator at 31^2 (complex Ritz pairs among the kept
    ones): the kept Ritz values and the improved span agree with the oracle's."""
    from oracle.gmresdr import arnoldi_e
    N, k, m = 31, 8, 24
    top, oop = tg.Operator("exp2d", N, EX1), OOp(EXP2D, N, EX1)
    Y0 = gi.random_dense((oop.n, k), 54)
    Yo, th_o, eres_o, done_o, _ = arnoldi_e(oop.apply, Y0, m, cycles, 4)
    defl = top.defl_from_basis(cu(Y0.T.copy()), k)
    th, st = defl.improve(m, cycles, 4)
    assert st["cycles"] == done_o == cycles and defl.kk == Yo.shape[1]
    assert np.max(np.abs(np.sort_complex(th) - np.sort_complex(th_o))) <= 1e-8 * np.max(np.abs(th_o))
    Yg = host(defl.copy(0)).T
    Qa, Qb = np.linalg.qr(Yo)[0], np.linalg.qr(Yg)[0]
    c = np.clip(np.linalg.svd(Qa.T @ Qb, compute_uv=False), 0, 1)
    assert np.max(np.sqrt(1 - c ** 2)) <= 1e-6


def test_arnoldi_e_improves_moved_vectors(tg):
    """The phase-2 use: coarse vectors moved to the fine grid, improved by Arnoldi-E until
    the 6 smallest pairs reach residual 1e-2 |theta| (the moved vectors start near 1, the
    oracle's run needs about 10 cycles); the two-grid solve still reaches the direct
    solution."""
    N = 127
    top, oop = tg.Operator("exp2d", N, EX1), OOp(EXP2D, N, EX1)
    b = gi.rhs(oop.n, 55)
    bt = cu(b)
    xc, defl, _, _ = top.coarse_gmresdr(bt, 40, 20, rtolev=1e-3, rtol=1e-8)
    th, st = defl.improve(50, 30, 6, nev=6, rtolev=1e-2)
    assert st["eig_converged"] >= 6 and 3 <= st["cycles"] < 30
    x = top.prolong(xc)
    status, s2 = top.solve(bt, x, defl, rtol=1e-10, ncyc=20, restart_mvps=0)
    assert status == tg.TG_OK
    assert rel(host(x), twogrid.exact_solution(oop, b)) <= 1e-6


def test_cubic_interpolation_moves_better_eigenvectors(tg):
    """The reason for the cubic reading: on the Helmholtz operator -Lap u - 30^2 u (127^2,
    coarse 63^2) the coarse GMRES-DR basis moved by cubic interpolation gives fine-grid Ritz
    pairs (Rayleigh-Ritz of A on the moved span, computed here with the oracle's operator)
    whose residuals ||A y - theta y|| / ||y||, for the 10 values nearest zero, are well
    below those of the bilinear move of the same coarse basis."""
    N, mass = 127, -900.0
    oop = OOp(CD2D, N, (0.0,), mass=mass)
    b = gi.rhs(oop.n, 45)
    med = {}
    for interp in ("linear", "cubic"):
        top = tg.Operator("cd2d", N, (0.0,), mass=mass, interp=interp)
        _, defl, _, _ = top.coarse_gmresdr(cu(b), 60, 30, rtolev=1e-8, rtol=1e-10, max_cycles=300, want_xc=False)
        Y = host(defl.copy(0)).reshape(defl.kk, oop.n).T
        Q = np.linalg.qr(Y)[0]
        AQ = np.stack([oop.apply(Q[:, j]) for j in range(Q.shape[1])], axis=1)
        theta, G = np.linalg.eig(Q.T @ AQ)
        near = np.argsort(np.abs(theta))[:10]
        res = [np.linalg.norm(AQ @ G[:, i] - theta[i] * (Q @ G[:, i])) / np.linalg.norm(G[:, i]) for i in near]
        med[interp] = float(np.median(res))
    assert med["cubic"] < 0.5 * med["linear"], med
