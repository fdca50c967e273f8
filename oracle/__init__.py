"""Plain FP64 CPU oracle for the two-grid deflated Krylov method (Morgan, Whyte, Wilcox,
Yang: "Two-grid deflated Krylov methods for linear equations").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or run this
package: only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
It shares no code with the CUDA library; the two meet only through the seeded inputs
of ``tg_inputs``.

Everything here is written for a reader checking it against the paper: numpy/scipy
FP64, no blocking, fusion or reordering beyond what the algorithms state; library
primitives (sparse matrix products, QR, eig, LU) serve as single steps.

Modules:
  operators  - the fine/coarse discrete operators (constant- and variable-coefficient
               convection-diffusion, 4D U(1) lattice) as matrix-free applies and as
               sparse matrices, and their transposes.
  transfer   - grid transfer: bilinear/trilinear prolongation, full-weighting
               restriction, the 2^4 block-transport prolongation of the lattice.
  krylov     - projections (Galerkin and MinRes, Section 2.2), restarted BiCGStab
               cycles and the BiCGStab(ncyc)-Proj(k) driver (Section 4.1), GMRES cycles
               and GMRES(m)-Proj(k) (Section 2.2).
  gmresdr    - GMRES-DR(m,k) with harmonic Ritz restarts (Section 2.1).
  adjoint    - adjoint solve and the kappa gradient of L = 1/2 ||x - x*||^2.

Pins (what ties each part to the paper or to mathematics rather than to itself) live
in tests/test_oracle_*.py.  Parity unpinned: the iteration counts of the iterative
methods (they depend on rounding), see the test headers.
"""
