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
    """Central differences of L with respect to kappa at the given flat node indices."""
    out = []
    for p in nodes:
        dk = rel_step * op.kappa[p]
        vals = []
        for sgn in (+1, -1):
            kap = op.kappa.copy()
            kap[p] += sgn * dk
            o2 = Operator(VARK2D, op.N, op.beta, kap)
            x = solve(o2, b)
            vals.append(0.5 * float((x - xstar) @ (x - xstar)))
        out.append((vals[0] - vals[1]) / (2 * dk))
    return np.array(out)
