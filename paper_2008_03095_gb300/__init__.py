"""GB300 (sm_103a) fused-sampling influence maximization (INFuseR-MG hot path,
arXiv 2008.03095) behind a small C ABI (include/im.h).

The Python names mirror the C entry points; all computation runs in the CUDA
library built by `paper_2008_03095_gb300.build.build()`.
"""
from ._binding import (IM_EBUSY, IM_ECUDA, IM_EINTERNAL, IM_EINVAL, IM_ENOMEM, IM_ETIMEOUT,
                       IM_OK, Graph, IMError, Workspace, header_functions,
                       im_debug_edge_hash, im_debug_estimate_spread_masked, im_debug_labels,
                       im_debug_lane_randoms, im_debug_select_seeds_masked, im_debug_sizes,
                       im_debug_tables_lanes, im_debug_override, im_debug_clear_overrides, im_debug_first_gains,
                       IM_OVR_CELF_CLUSTER, IM_OVR_CELF_ROUND_CAP, IM_OVR_UF_CAP,
                       IM_OVR_SPREAD_LEVEL_CAP, IM_OVR_FAIL_ALLOC, IM_OVR_CELF_REFRESH_AFTER, IM_OVR_BATCH_GROUP,
                       IM_OVR_CELF_EXT_REFRESH,
                       IM_NUM_OVERRIDES, IM_SAMPLE_EDGE_WEIGHTS, IM_SAMPLE_MIXED_HASH,
                       IM_ALGO_FUSED_SAMPLING, im_graph_create_weighted, im_select_seeds_ex,
                       im_estimate_spread_ex, im_select_seeds_ex_async,
                       im_estimate_spread_ex_async, im_debug_tables_ex, Batch, BatchQuery,
                       im_batch_create, im_batch_run_async, im_batch_results,
                       im_batch_query_stats, im_batch_info, im_batch_autotune,
                       im_batch_destroy, im_batch_phase_cycles, BATCH_PHASES, im_autotune_cache_save, im_autotune_cache_load,
                       im_autotune_cache_clear, BATCH_INFO, Server, Request,
                       IM_REQUEST_SELECT, IM_REQUEST_SPREAD, im_server_create, im_server_submit,
                       im_server_wait, im_server_stats, im_server_destroy, SERVER_STATS,
                       im_estimate_spread, im_estimate_spread_async, im_estimate_spread_noalloc,
                       im_graph_create, NOALLOC_LIMITS,
                       im_graph_create_raw, im_graph_destroy, im_graph_info, im_kernel_launches,
                       im_last_error, im_profile_enable, im_profile_read, PHASES,
                       im_sampling_threshold, im_select_seeds, im_select_seeds_async,
                       im_set_stream, im_workspace_create, im_workspace_destroy,
                       im_workspace_stats, im_workspace_status, lib, library_path, STATS)
