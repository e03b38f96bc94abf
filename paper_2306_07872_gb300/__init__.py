"""GB300-native (sm_103a) weighted DAWN: GOVM shortest paths behind a C ABI.

The compute path is libdawn.so (CUDA kernels for sm_103a, declared in
include/dawn.h); :mod:`paper_2306_07872_gb300.dawn` is its thin binding.
"""
from .dawn import (  # noqa: F401
    DAWN_ERR_BOUNDS, DAWN_ERR_CUDA, DAWN_ERR_INVALID, DAWN_ERR_NOT_CONVERGED, DAWN_ERR_OOM, DAWN_ERR_TIMEOUT, DAWN_OK,
    DAWN_FRONTIER_AUTO, DAWN_FRONTIER_BITMAP, DAWN_FRONTIER_QUEUE, DAWN_OPT_FRONTIER, DAWN_OPT_SKIP_REMARKED,
    DAWN_OPT_BATCH, DAWN_OPT_CTAS_PER_SM, DAWN_OPT_GRID_BLOCKS, DAWN_OPT_GSVM, DAWN_OPT_MAX_STEPS, DAWN_OPT_SMALL_PATH, DAWN_OPT_TEST_FAIL_ALLOC, DAWN_OPT_TEST_STALL, DAWN_SMALL_AUTO, DAWN_SMALL_NEVER,
    DAWN_SMALL_WHEN_STATE_FITS,
    DAWN_OPT_TRACE_STEPS, DAWN_OPT_WAIT_LIMIT_NS, DAWN_TUNE_MSSSP, DAWN_TUNE_ROOTS, DAWN_TUNE_SSSP, DAWN_W_F32, DAWN_W_I32,
    DAWN_W_U32, DAWN_WEIGHTS_DEFER_CHECK, DAWN_WEIGHTS_ON_DEVICE, EXPORTS, DawnError, DawnSSSP, Graph, dawn_autotune, dawn_create_graph, dawn_destroy, dawn_get_stats,
    dawn_get_trace, dawn_graph_info, dawn_msssp,
    dawn_reserve, dawn_set_option, dawn_set_weights, dawn_sssp, dawn_sssp_backward, dawn_sssp_noalloc, dawn_sssp_roots, dawn_status,
    dawn_status_string, dawn_trim_memory, load_library,
)
