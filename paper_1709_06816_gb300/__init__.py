"""GB300-native Lance-Williams agglomerative clustering.

The hot path -- all n - 1 merges of Section 4's iteration (minimum search, combine,
update with the Table 1 coefficients, output) -- runs in hand-written CUDA
kernels for sm_103a inside ``liblw.so``; this package only builds the library
and marshals arguments to its C ABI (``include/lw.h``).
"""
from .native import (  # noqa: F401
    Context,
    LwError,
    LINKAGES,
    LW_SINGLE,
    LW_COMPLETE,
    LW_AVERAGE,
    LW_WARD,
    LW_WEIGHTED,
    LW_CENTROID,
    lw_create,
    lw_cluster,
    lw_cluster_async,
    lw_wait,
    lw_get_stats,
    lw_set_option,
    lw_status_string,
    lw_destroy,
)
