"""Stable-vertex-value queries over evolving graphs on GB300 (sm_103a).

The compute path lives in ``libsvv.so`` (CUDA kernels behind the C ABI of
``include/svv.h``); ``svv`` is its ctypes binding.
"""
from .svv import (SVV_BFS, SVV_SSNP, SVV_SSSP, SVV_SSWP, Context, SvvError, lib, svv_build_versioned_csr,  # noqa: F401
                  svv_create, svv_destroy, svv_device_bytes, svv_get_bounds, svv_get_stats, svv_last_error, svv_load,
                  svv_query, svv_query_batch, svv_query_compact, svv_query_host, svv_query_plain, svv_set_tuning, svv_status_str, to_u32,
                  svv_serve_start, svv_autotune, svv_submit, svv_poll, svv_ticket_info, svv_release, svv_serve_stop)
