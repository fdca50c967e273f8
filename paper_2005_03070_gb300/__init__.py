"""GB300 (sm_103a) two-grid deflated Krylov solver: coarse GMRES-DR eigenvectors, moved to
the fine grid, deflating restarted BiCGStab / GMRES through projections between cycles.

The compute path is libtg.so (CUDA kernels + C ABI, include/tg.h); ``tg`` is its thin
ctypes binding.  Build with ``python -m paper_2005_03070_gb300.build``.
"""
from . import tg  # noqa: F401
from .tg import Deflation, Operator, harmonic_ritz, load  # noqa: F401
