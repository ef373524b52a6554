"""GB300-native generalized-random-tree point solver (arXiv 2402.06491).

The product is the C-ABI library libgrt.so (include/grt.h) built from
``csrc/`` for sm_103a; this package holds its ctypes binding (same names as
the C calls), its build step and the host-side sharding of points over ranks.
"""
from ._binding import (  # noqa: F401
    EXPORTED, GrtError, Context, Plan, Server, grt_poll, grt_poll_ex, grt_cancel, grt_server_create, grt_server_destroy, grt_server_sizes,
    grt_server_last_error, grt_server_stats, grt_submit, grt_create, grt_destroy, grt_last_error, grt_pade, grt_pade_error, grt_plan_counters, grt_plan_kappa,
    grt_plan_autotune, grt_plan_create, grt_plan_destroy, grt_plan_get_config, grt_plan_graph_capture,
    grt_plan_graph_launch, grt_pdd_points, grt_pdd_solve, grt_pdd_solve_range, grt_spline_grid, pdd_grid_struct, grt_plan_set_config, grt_set_solve_config, grt_plan_execute, grt_plan_launches, grt_plan_set_timing, grt_plan_timing, grt_solve, grt_solve_noalloc, grt_solve_plain, grt_trees, library_path,
    problem_struct, NOALLOC_MAX_POINTS, NOALLOC_MAX_TREES, STATUS_HIGH_PRUNE, STATUS_PADE_POLE_NEAR, STATUS_PADE_SINGULAR, STATUS_SERIES_PARTIAL,
)
from .sharding import pdd_subdomain_range, shard_range  # noqa: F401
