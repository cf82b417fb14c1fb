"""GB300 (sm_103a) implementation of the diffusion operator of the
splitting-free vorticity redistribution method (Kirchhart & Obi,
arXiv 1508.06379).

The compute path is the CUDA library libvrm.so (C ABI in include/vrm.h);
this package holds its build and a thin ctypes binding with the same names
as the C entry points.
"""
from .binding import (KCAP_MAX, LP_FULL, LP_LEARNED, LP_NONE, LP_NOT_DIFFUSED, LP_SMALL, learned_targets, STENCIL_W, STENCIL_W2, VRM, VRM_ERR_ARG,
                      VRM_ERR_CAPACITY, VRM_ERR_CUDA, VRM_ERR_UNSUPPORTED, VRM_OK, Params, Stats, VRMError,
                      library_path, load_library, launch_count, STAGES, build_neighbourhoods_noalloc, fma_peak,
                      NOALLOC_MAX_N, VRMBatch, Cloud, Schedule, MLP, MLP_PARAMS, MLP_IN, MLP_OUT)
from .builder import build

__all__ = ["VRM", "VRMBatch", "Cloud", "Schedule", "MLP", "MLP_PARAMS", "MLP_IN", "MLP_OUT", "VRMError", "Params", "Stats", "build", "load_library", "library_path", "launch_count", "STAGES",
           "build_neighbourhoods_noalloc", "fma_peak", "NOALLOC_MAX_N", "STENCIL_W", "STENCIL_W2", "KCAP_MAX",
           "LP_NOT_DIFFUSED", "LP_SMALL", "LP_FULL", "LP_NONE", "LP_LEARNED", "learned_targets", "VRM_OK", "VRM_ERR_ARG", "VRM_ERR_CAPACITY",
           "VRM_ERR_CUDA", "VRM_ERR_UNSUPPORTED"]
