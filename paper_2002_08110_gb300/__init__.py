"""GB300-native (sm_103a) matrix-free DG advection in 2 to 6 dimensions.

The method is that of hyper.deal (Munch, Kormann & Kronbichler, arXiv
2002.08110): the upwind discontinuous Galerkin advection operator on the
tensor product of a configuration-space and a velocity-space mesh, evaluated
element by element with sum factorisation, inside low-storage Runge-Kutta
time stepping.  The work runs in the CUDA library ``libdg.so`` behind the C
ABI of ``include/dg.h``; this package is its thin Python binding plus the
autograd wrapper of the adjoint.
"""
from ._lib import (BASIS_GL, BASIS_GLL, BASIS_GLL_GAUSS, PREC_FP32, PREC_FP64,  # noqa: F401
                   PREC_MIXED, DGError)

__all__ = ["DG", "DGBatch", "DGError", "PREC_FP64", "PREC_FP32", "PREC_MIXED", "BASIS_GL",
           "BASIS_GLL", "BASIS_GLL_GAUSS", "reference_nodes", "basis_nodes", "build_library"]


def build_library(verbose=False):
    from .build import build
    return build(verbose=verbose)


def __getattr__(name):
    # torch-dependent parts are imported lazily
    if name in ("DG", "DGBatch", "reference_nodes", "basis_nodes", "from_spec"):
        from . import api
        return getattr(api, name)
    if name in ("RKForward", "final_state", "misfit_gradient", "CheckpointMismatch"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
