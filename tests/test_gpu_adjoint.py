"""The differentiable solve at full size: 511^2 variable-coefficient
convection-diffusion, kappa = exp(GRF) (length scale 0.1, sigma = 1), beta = 1, coarse
255^2 with 20 left eigenvectors, float32 inner / float64 refinement both ways.

dL/dkappa for L = 1/2 ||x - x*||^2 (x* ~ N(0,1), seeded) from the autograd wrapper must
match (a) the oracle's gradient from direct solves, relative 1e-5 in norm, and (b)
central finite differences of direct solves on 64 seeded interior kappa nodes, relative
1e-5, plus the recompute-x variant."""
import numpy as np
import pytest

import tg_inputs as gi
from oracle import adjoint
from oracle.operators import VARK2D, Operator as OOp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 511


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_03070_gb300 import build
    build.build()
    kap = gi.kappa_grf(N, 0)
    n = N * N
    b = gi.rhs(n, 0)
    xstar = gi.random_dense(n, 11)
    oop = OOp(VARK2D, N, (1.0,), kap)
    Lo, grad_o, x_o, lam_o = adjoint.loss_and_gradient(oop, b, xstar)
    return kap, b, xstar, oop, Lo, grad_o


def _gpu_grad(kap, b, xstar, recompute):
    from paper_2005_03070_gb300.autograd import two_grid_solve
    kt = torch.from_numpy(kap).cuda().requires_grad_(True)
    bt = torch.from_numpy(b).cuda()
    xs = torch.from_numpy(xstar).cuda()
    x = two_grid_solve(kt, bt, N, beta=1.0, m=40, k=20, rtolev=1e-2, rtol=1e-11, ncyc=20, precision="f32_ir",
                       recompute=recompute)
    L = 0.5 * torch.sum((x - xs) ** 2)
    L.backward()
    torch.cuda.synchronize()
    return float(L.item()), kt.grad.detach().cpu().numpy(), x.detach().cpu().numpy()


def test_adjoint_gradient_full_size(setup):
    kap, b, xstar, oop, Lo, grad_o = setup
    L, g, x = _gpu_grad(kap, b, xstar, recompute=False)
    assert np.linalg.norm(b - oop.apply(x)) / np.linalg.norm(b) <= 1e-11
    assert abs(L - Lo) <= 1e-9 * abs(Lo)
    assert np.linalg.norm(g - grad_o) / np.linalg.norm(grad_o) <= 1e-5
    nodes = gi.kappa_fd_nodes(N, 64, 0)
    fd = adjoint.finite_difference(oop, b, xstar, nodes)
    scale = np.abs(fd).max()
    assert np.max(np.abs(g[nodes] - fd) / np.maximum(np.abs(fd), 1e-3 * scale)) <= 1e-5


def test_adjoint_recompute_matches(setup):
    kap, b, xstar, oop, Lo, grad_o = setup
    _, g, _ = _gpu_grad(kap, b, xstar, recompute=True)
    assert np.linalg.norm(g - grad_o) / np.linalg.norm(grad_o) <= 1e-5
