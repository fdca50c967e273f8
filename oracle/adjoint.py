"""Adjoint solve and the gradient of L = 1/2 ||x - x*||^2 with respect to the node
diffusion field kappa of the variable-coefficient operator, FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Not in the paper (an added differentiable form of its solve).  Derivation: A(kappa) x = b
gives dx = -A^{-1} (dA) x, so dL = (x - x*)^T dx = -lambda^T (dA) x with A^T lambda = g,
g = x - x*.  The diffusion part of lambda^T A x is
  sum over faces f = (a, b) of kappa_f (lambda_a - lambda_b)(x_a - x_b) / h^2,
kappa_f = (kappa_a + kappa_b) / 2, with lambda = x = 0 on the boundary nodes, so
  dL/dkappa_p = -1/2 sum_{faces f touching p} (lambda_a - lambda_b)(x_a - x_b) / h^2.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .operators import VARK2D, Operator


def solve(op: Operator, b):
    return spla.spsolve(op.sparse().tocsc(), b)


def solve_transposed(op: Operator, g):
    """lambda = A^{-T} g by sparse LU of the assembled A^T (not the beta-negation shortcut)."""
    return spla.spsolve(op.sparse().T.tocsc(), g)


def kappa_gradient(op: Operator, x, lam) -> np.ndarray:
    """dL/dkappa on all (N+2)^2 nodes from x and the adjoint lambda (face by face)."""
    assert op.kind == VARK2D
    N = op.N
    h = 1.0 / (N + 1)
    X = np.zeros((N + 2, N + 2))
    Lm = np.zeros((N + 2, N + 2))
    X[1:-1, 1:-1] = x.reshape(N, N)
    Lm[1:-1, 1:-1] = lam.reshape(N, N)
    grad = np.zeros((N + 2, N + 2))
    # horizontal faces between (j, i) and (j, i+1), i = 0..N, j = 1..N (at least one interior node)
    fh = -(Lm[1:-1, :-1] - Lm[1:-1, 1:]) * (X[1:-1, :-1] - X[1:-1, 1:]) / h**2
    grad[1:-1, :-1] += 0.5 * fh
    grad[1:-1, 1:] += 0.5 * fh
    # vertical faces between (j, i) and (j+1, i), j = 0..N, i = 1..N
    fv = -(Lm[:-1, 1:-1] - Lm[1:, 1:-1]) * (X[:-1, 1:-1] - X[1:, 1:-1]) / h**2
    grad[:-1, 1:-1] += 0.5 * fv
    grad[1:, 1:-1] += 0.5 * fv
    return grad.reshape(-1)


def loss_and_gradient(op: Operator, b, xstar):
    """L(kappa) and dL/dkappa by direct solves (the plain definition)."""
    x = solve(op, b)
    g = x - xstar
    lam = solve_transposed(op, g)
    return 0.5 * float(g @ g), kappa_gradient(op, x, lam), x, lam


def finite_difference(op: Operator, b, xstar, nodes, rel_step=1e-4):
    """Central differences (L(kappa + h e_p) - L(kappa - h e_p)) / 2h at the given flat node
    indices, h = rel_step * kappa_p.

    L is of order n while its change is of order h |dL/dkappa_p|, so subtracting two
    separately computed losses cancels most digits.  The difference is formed instead
    from the change of the solution: x_pm = x + d_pm with A(kappa_pm) d_pm = b - A(kappa_pm) x,
    and L_pm - L = g^T d_pm + 1/2 ||d_pm||^2 with g = x - x* (identities, no truncation).
    d_pm is solved by refinement with the sparse LU of the unperturbed A (A(kappa_pm) - A
    is of relative size rel_step, so each step gains about -log10(rel_step) digits); the
    loop stops on the residual of the perturbed system itself."""
    lu = spla.splu(op.sparse().tocsc())
    x = lu.solve(b)
    g = x - xstar
    out = []
    for p in nodes:
        dk = rel_step * op.kappa[p]
        dL = []
        for sgn in (+1, -1):
            kap = op.kappa.copy()
            kap[p] += sgn * dk
            Ap = Operator(VARK2D, op.N, op.beta, kap)
            rhs = b - Ap.apply(x)
            d = np.zeros_like(x)
            for _ in range(50):
                res = rhs - Ap.apply(d)
                if np.linalg.norm(res) <= 1e-15 * np.linalg.norm(rhs):
                    break
                d += lu.solve(res)
            else:
                raise RuntimeError("finite_difference: refinement did not converge")
            dL.append(float(g @ d) + 0.5 * float(d @ d))
        out.append((dL[0] - dL[1]) / (2 * dk))
    return np.array(out)
