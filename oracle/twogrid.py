"""Two-grid deflated BiCGStab / GMRES (Sections 3 and 4.1), FP64, and the plain
definition x* = A^{-1} b used as the end-to-end parity target.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Phases (Section 3 box, Section 4.1 box):
  1. GMRES-DR(m,k) on the coarse grid (coarse right-hand side b_c = R b, full weighting;
     lattice: b_c = P^H b), giving x_c and the k approximate eigenvectors;
     they are moved to the fine grid by the prolongation P; x0 = P x_c.
  2. (Arnoldi-E improvement: not part of this path.)
  3. BiCGStab(ncyc)-Proj(k) or GMRES(m3)-Proj(k) on the fine grid.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse.linalg as spla

from . import krylov, transfer
from .gmresdr import gmresdr
from .operators import CD2D, CD3D, EXP2D, U1_4D, VARK2D, Operator, coarse_operator


@dataclass
class CoarseLevel:
    op_c: Operator | None
    apply_c: object
    prolong: object          # coarse vector -> fine vector
    restrict: object         # fine vector -> coarse vector
    n_c: int


def coarse_level(op: Operator) -> CoarseLevel:
    if op.kind in (CD2D, VARK2D, EXP2D):
        opc = coarse_operator(op)
        return CoarseLevel(opc, opc.apply, lambda v: transfer.prolong2d(v, opc.N),
                           lambda v: transfer.restrict(v, op.N, 2), opc.n)
    if op.kind == CD3D:
        opc = coarse_operator(op)
        return CoarseLevel(opc, opc.apply, lambda v: transfer.prolong3d(v, opc.N),
                           lambda v: transfer.restrict(v, op.N, 3), opc.n)
    Ac, P, *_ = transfer.lattice_coarse_stencil(op)
    return CoarseLevel(None, lambda v: Ac @ v, lambda v: P @ v, lambda v: P.conj().T @ v,
                       Ac.shape[0])


def exact_solution(op: Operator, b: np.ndarray) -> np.ndarray:
    """x* = A^{-1} b by sparse LU (the plain definition of what the solve converges to)."""
    return spla.spsolve(op.sparse().tocsc(), b)


@dataclass
class TwoGridResult:
    x: np.ndarray
    solve: krylov.SolveResult
    coarse: object
    Y: np.ndarray
    x0: np.ndarray


def two_grid_solve(op: Operator, b, m=30, k=15, nev=None, rtolev=1e-6, rtol_c=1e-8,
                   max_cycles=300, method="bicgstab", proj="minres", rtol=1e-8, ncyc=0,
                   restart_mvps=60, m3=20, max_mvps=100000, level: CoarseLevel | None = None):
    level = coarse_level(op) if level is None else level
    bc = level.restrict(b)
    gd = gmresdr(level.apply_c, bc, m, k, nev=nev, rtolev=rtolev, rtol=rtol_c,
                 max_cycles=max_cycles, dtype=op.dtype)
    Y = np.stack([level.prolong(gd.Yc[:, j]) for j in range(gd.Yc.shape[1])], axis=1)
    x0 = level.prolong(gd.x)
    defl = krylov.make_deflation(op.apply, Y, proj)
    if method == "bicgstab":
        res = krylov.bicgstab_proj(op.apply, b, x0, defl, rtol=rtol, ncyc=ncyc,
                                   restart_mvps=restart_mvps, max_mvps=max_mvps)
    else:
        res = krylov.gmres_proj(op.apply, b, x0, defl, m=m3, rtol=rtol, max_mvps=max_mvps)
    return TwoGridResult(res.x, res, gd, Y, x0)
