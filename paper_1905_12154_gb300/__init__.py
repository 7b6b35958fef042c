"""GB300-native back-and-forth method for quadratic-cost optimal transport.

The method of Jacobs & Leger (arXiv 1905.12154), Algorithm 1 with the step
rule of Section 4.2, runs in the CUDA library ``libbfm.so`` (sm_103a) behind
the C ABI of ``include/bfm.h``; ``binding`` is a thin ctypes layer over it
whose functions carry the C names.  Importing the package does not load the
library; the first call does, and fails loudly if it was not built.
"""
from .binding import (  # noqa: F401
    BFM_FP32, BFM_FP64, BFM_OK, BFM_NOT_CONVERGED, BfmError,
    bfm_ctransform, bfm_interpolate, bfm_map, bfm_poisson, bfm_pushforward,
    bfm_solve, bfm_solve_host, bfm_workspace_bytes, bfm_workspace_bytes_host,
    bfm_poisson_workspace_bytes, status_string, last_error, bfm_solve_batched,
    bfm_w2_backward, w2_loss, BfmSolver,
)
