"""GPU parity at the full sizes of the benchmarked workloads, where the kernels take code
paths that small grids never reach (through the C ABI).

At 255^3 (16,581,375 unknowns) a grid-stride launch of 8 blocks of 256 threads per SM gives
every thread about 53 passes; the pipelined V^H w on the 127^3 coarse grid (2,048,383 rows)
walks about 32,000 chunks of 64 float64 (or 16,000 of 128 float32) rows over at most 2 blocks
per SM, wrapping its 3-stage cp.async ring thousands of times.  The batched form is run
on instances of 255^2, 511^2 and 1023^2 (the range of the batched workload).

Bars: per operator application <= 1e-13 relative in float64 and <= 1e-6 in float32; one
GMRES-DR cycle (= GMRES(m)) gives the oracle's coarse solution to 1e-10 (float64 basis) and
1e-4 (float32 basis); a 12-product BiCGStab cycle gives the oracle's iterate to 1e-11
(float64) and 1e-5 (float32 inner cycle added to the float64 x); the batched solutions
reach rtol = 1e-10 by the oracle's operator and the sparse-LU solution to 1e-6.
"""
import numpy as np
import pytest

import tg_inputs as gi
from oracle import krylov, transfer
from oracle.gmresdr import gmresdr
from oracle.operators import CD2D, CD3D, Operator as OOp, coarse_operator

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BETA3 = (2.0, 1.0, 0.5)


@pytest.fixture(scope="module")
def tg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_03070_gb300 import build
    build.build()
    from paper_2005_03070_gb300 import tg as mod
    mod.load()
    return mod


@pytest.fixture(scope="module")
def cd3d_255(tg):
    return tg.Operator("cd3d", 255, BETA3), OOp(CD3D, 255, BETA3)


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_apply_255(tg, cd3d_255):
    top, oop = cd3d_255
    u = gi.rhs(oop.n, 31)
    ref = oop.apply(u)
    y = host(top.apply(cu(u)))
    assert rel(y, ref) <= 1e-13
    assert np.max(np.abs(y - ref)) <= 1e-13 * np.max(np.abs(ref))
    yt = host(top.apply(cu(u), transpose=True))
    assert rel(yt, oop.transposed().apply(u)) <= 1e-13
    y32 = host(top.apply(cu(u.astype(np.float32)), precision=tg.TG_F32_IR)).astype(np.float64)
    assert rel(y32, ref) <= 1e-6


@pytest.mark.parametrize("precision,tol", [("f64", 1e-10), ("f32_ir", 1e-4)])
def test_coarse_gmres_cycle_127(tg, cd3d_255, precision, tol):
    top, oop = cd3d_255
    opc = coarse_operator(oop)
    b = gi.rhs(oop.n, 32)
    bc = transfer.restrict_stencil(b, 255, 3)
    m, k = 12, 4
    ref = gmresdr(opc.apply, bc, m, k, rtolev=1e-12, rtol=1e-14, max_cycles=1)
    xc, _, st, _ = top.coarse_gmresdr(cu(b), m, k, rtolev=1e-12, rtol=1e-14, max_cycles=1, precision=precision,
                                      want_defl=False)
    assert st["cycles"] == 1
    assert rel(host(xc), ref.x) <= tol


def test_bicgstab_12_products_255(tg, cd3d_255):
    top, oop = cd3d_255
    b = gi.rhs(oop.n, 33)
    x0 = np.zeros(oop.n)
    ref = krylov.bicgstab_proj(oop.apply, b, x0, None, rtol=1e-14, ncyc=0, restart_mvps=12, max_mvps=12)
    assert ref.mvps == 12
    for precision, tol in (("f64", 1e-11), ("f32_ir", 1e-5)):
        xt = cu(x0.copy())
        st, stats = top.solve(cu(b), xt, rtol=1e-14, ncyc=0, restart_mvps=12, max_mvps=12, precision=precision)
        assert stats[0]["mvps"] == 12
        assert rel(host(xt), ref.x) <= tol, precision


def test_batch_full_range_sizes(tg):
    import scipy.sparse.linalg as spla
    Ns, betas = [255, 1023, 511], [0.5, 2.0, 4.0]
    batch = tg.Batch(Ns, betas)
    blocks = []
    for i, N in enumerate(Ns):
        B = gi.rhs(N * N, seed=200 + i, nrhs=8)
        blocks.append(np.ascontiguousarray(B.T).reshape(-1))
    rhs = cu(np.concatenate(blocks))
    batch.setup(rhs, m=40, k=20, rtolev=1e-2, threads=3)
    x = torch.zeros_like(rhs)
    status, stats = batch.solve(rhs, x, rtol=1e-10, ncyc=20, restart_mvps=0, threads=3)
    assert status == tg.TG_OK, [s["status"] for s in stats]
    xh = host(x)
    for i, N in enumerate(Ns):
        op = OOp(CD2D, N, (betas[i],))
        lu = spla.splu(op.sparse().tocsc())
        o, n = batch.offsets[i], batch.sizes[i]
        B = blocks[i].reshape(n, 8)
        X = xh[o:o + n * 8].reshape(n, 8)
        for q in range(8):
            b, xq = B[:, q], X[:, q]
            assert np.linalg.norm(b - op.apply(xq)) / np.linalg.norm(b) <= 1e-10
            xs = lu.solve(b)
            assert rel(xq, xs) <= 1e-6
