"""GB300-native patchy semi-Lagrangian solver for minimum-time HJB equations.

A thin ctypes binding over ``libhjbp.so`` (C ABI in ``include/hjbp.h``).  Every
step of a solve runs in the library's CUDA kernels; this module only marshals
arguments.  There is no CPU fallback: if the library is missing the first call
raises.
"""
from ._binding import (  # noqa: F401
    HJBP_FP32_POLISH64,
    HJBP_FLAG_CAUSAL_SWEEPS,
    HJBP_FLAG_DIRICHLET,
    HJBP_FLAG_TILE_QUEUE,
    HJBP_FLAG_TIME_SWEEPS,
    HJBP_FLAG_WARM_START,
    HJBP_FP64,
    HJBP_OUT_ASTAR,
    HJBP_OUT_PHI,
    HJBP_OUT_U0,
    HJBP_OUT_U32,
    HJBP_OUT_UCOARSE,
    HjbpError,
    Plan,
    Stats,
    desc_from_problem,
    hjbp_batch_solve,
    hjbp_create,
    hjbp_destroy,
    hjbp_get_device_views,
    hjbp_get_intermediate,
    hjbp_get_labels,
    hjbp_get_sizes,
    hjbp_get_stats,
    hjbp_get_values,
    hjbp_last_error,
    hjbp_set_initial,
    hjbp_solve,
    hjbp_sync,
    hjbp_solve_global2d_noalloc,
    HJBP_NOALLOC_MAX_NODES,
    hjbp_server_create,
    hjbp_server_destroy,
    hjbp_server_poll,
    hjbp_server_stats,
    hjbp_server_submit,
    hjbp_version,
    library,
    library_path,
    torch_allocator,
)
