"""GB300 (sm_103a) deflated multigrid multilevel Monte Carlo for tr(D^{-1}) of
the 2D Wilson-Schwinger operator (Frommer & Ramirez-Hidalgo, Lattice 2022).

The computation lives in ``libmgmlmc.so`` (CUDA kernels behind the C ABI of
``include/mgmlmc.h``); ``Context`` and ``Server`` are its thin Python binding.
"""
from ._lib import (Context, MgmlmcError, Options, Server, default_options, estimate_concurrent,  # noqa: F401
                   estimate_trace_concurrent, fma_peak, load, make_request, request_footprint, LIB_PATH,
                   ECANCELLED, PENDING, OP_D, OP_PH, OP_P, OP_G5, OP_PREC, OP_DINV_C, OP_SMOOTH)
