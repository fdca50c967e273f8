"""GPU parity of the BiCGStab(ncyc)-Proj(k) cycle schedule (Section 4.1, steps 3a-3d).

The library's per-cycle history (||r|| / ||b|| after the step-3a projection, the step-3b
tolerance rticyc, products so far) is compared cycle by cycle with the oracle's
bicgstab_proj on the same inputs: the oracle's own coarse GMRES-DR basis and coarse
solution, prolonged by the oracle, are handed to both sides (so nothing on the oracle's
side comes from the CUDA path).

Bars: the number of cycles and the products per cycle are integers decided in float64 on
both sides, so they must agree exactly; ||r|| / ||b|| and rticyc agree to 1e-6 relative
(the two BiCGStab runs differ only by summation order, which hundreds of products
amplify well below that).  The reading past ncyc (cycles aiming at rtol ||b|| / ||r||
until convergence) is exercised by a schedule whose capped cycles cannot finish within
ncyc.
"""
import numpy as np
import pytest

import tg_inputs as gi
from oracle import krylov
from oracle.gmresdr import gmresdr
from oracle.operators import CD2D, Operator as OOp, coarse_operator
from oracle import transfer

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


def _oracle_inputs(N, beta, m, k, seed):
    oop = OOp(CD2D, N, beta)
    opc = coarse_operator(oop)
    b = gi.rhs(oop.n, seed)
    gd = gmresdr(opc.apply, transfer.restrict(b, N, 2), m, k, rtolev=1e-4, rtol=1e-8, max_cycles=300)
    Y = np.stack([transfer.prolong2d(gd.Yc[:, j], opc.N) for j in range(gd.Yc.shape[1])], axis=1)
    x0 = transfer.prolong2d(gd.x, opc.N)
    return oop, b, Y, x0


def _compare(ref, st, ncyc):
    h = st["history"]
    assert st["cycles"] == ref.cycles == len(ref.history) == len(h), (st["cycles"], ref.cycles)
    assert st["mvps"] == ref.mvps
    for c, ((icyc, relres_o, rt_o, mv_o), (relres_g, rt_g, mv_g)) in enumerate(zip(ref.history, h)):
        assert icyc == c + 1
        assert int(mv_g) == mv_o, (c, mv_g, mv_o)
        assert abs(relres_g - relres_o) <= 1e-6 * relres_o, (c, relres_g, relres_o)
        assert abs(rt_g - rt_o) <= 1e-6 * rt_o, (c, rt_g, rt_o)
        if ncyc and icyc > ncyc:
            # past ncyc: the cycle aims at rtol ||b|| / ||r||
            assert abs(rt_g * relres_g - 1e-8) <= 1e-8 * 1e-9


@pytest.mark.parametrize("N,ncyc,cap", [(127, 20, 0), (63, 3, 12)])
def test_cycle_history_matches_oracle(tg, N, ncyc, cap):
    oop, b, Y, x0 = _oracle_inputs(N, (1.0,), 30, 15, seed=21)
    defl_o = krylov.make_deflation(oop.apply, Y, "minres")
    ref = krylov.bicgstab_proj(oop.apply, b, x0, defl_o, rtol=1e-8, ncyc=ncyc,
                               restart_mvps=cap or None, max_mvps=100000)
    assert ref.converged
    top = tg.Operator("cd2d", N, (1.0,))
    defl = top.defl_from_basis(cu(Y.T.copy()), Y.shape[1])
    x = cu(x0.copy())
    status, stats = top.solve(cu(b), x, defl, rtol=1e-8, ncyc=ncyc, restart_mvps=cap, max_mvps=100000,
                              history=500)
    assert status == tg.TG_OK, stats
    _compare(ref, stats[0], ncyc)
    if cap:
        assert ref.cycles > ncyc           # the continuation past ncyc was exercised
