"""B300-native linear-BVH geometric search (ArborX, arXiv 1908.11807).

The compute path is the CUDA library ``libarborx_b300.so`` (sm_103a), reached
through its C ABI (``include/arborx_b300.h``); this package is the thin Python
binding over it.  PyTorch supplies device memory and streams only.
"""
from ._binding import (  # noqa: F401
    ARBORX_BOXES,
    ARBORX_BUILD_APETREI,
    ARBORX_BUILD_KARRAS,
    ARBORX_ECUDA,
    ARBORX_EINVAL,
    ARBORX_ENOMEM,
    ARBORX_EOVERFLOW,
    ARBORX_ESTATE,
    ARBORX_ETIMEOUT,
    ARBORX_MAX_K,
    ARBORX_OK,
    ARBORX_POINTS,
    ArborXError,
    MLP_PARAMS,
    BVH,
    Batch,
    batched,
    order,
    arborx_build,
    arborx_query_nearest,
    arborx_query_spatial,
    arborx_sort_pairs,
    default_opts,
    profile_enable,
    profile_report,
    release_cached_memory,
    error_string,
    lib,
    version,
    LIB_PATH,
)
