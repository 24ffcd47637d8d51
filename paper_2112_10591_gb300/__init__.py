"""GB300-native event-based optical flow (Brebion, Moreau, Davoine).

The compute lives in libebof.so (CUDA, sm_103a); ``binding`` exposes its C
ABI (include/ebof.h) under the same names.  ``synth`` draws the seeded
synthetic event streams used by the tests and the benchmark.
"""
from .binding import (  # noqa: F401
    EBOF_ERR_BUSY, EBOF_ERR_CUDA, EBOF_ERR_DEVICE_BOUNDS, EBOF_ERR_INVALID_ARG,
    EBOF_ERR_OOM, EBOF_ERR_TIMEOUT, EBOF_ERR_UNSUPPORTED, EBOF_NO_PREVIOUS, EBOF_OK,
    EbofError, Stream, check, ebof_alpha_from_dsat, ebof_default_params, ebof_edt,
    ebof_params, ebof_process_surface, ebof_process_window, ebof_process_window_host,
    ebof_process_window_host_async, ebof_process_window_async, ebof_stream_join,
    ebof_process_windows, ebof_status_string, ebof_stream_create, ebof_stream_destroy,
    ebof_stream_reset, ebof_stream_sync, ebof_window_stats, library_path, load,
    EBOF_STAGE_COUNT, ebof_kernel_launches, ebof_stage_name, ebof_stream_get_profile,
    ebof_stream_set_profiling, ebof_edt_static, ebof_stream_get_profile_level,
    EBOF_STORAGE_FP16, EBOF_STORAGE_FP32, Group, ebof_window_desc, ebof_group_create,
    ebof_group_reset, ebof_group_process, ebof_group_flow, ebof_group_sync,
    ebof_stream_device_bytes, ebof_process_window_list, EBOF_QUEUED, EBOF_ERR_CANCELLED,
    Server, ebof_completion, ebof_now_ns, ebof_server_close_stream, ebof_server_config,
    ebof_server_create, ebof_server_default_config, ebof_server_destroy, ebof_server_drain,
    ebof_server_get_info, ebof_server_info, ebof_server_open_stream, ebof_server_poll,
    ebof_server_submit, EBOF_SURFACE_EXP, EBOF_SURFACE_LINEAR, EBOF_SURFACE_BOUNDED,
    EBOF_SURFACE_LOG, ebof_fwl, ebof_fwl_scratch_bytes, ebof_stream_set_wait_limit,
    ebof_debug_fail_allocation, MultiGroup, ebof_multigroup_create, ebof_multigroup_process,
    ebof_multigroup_set_fused, ebof_stream_get_pyramid,
)
