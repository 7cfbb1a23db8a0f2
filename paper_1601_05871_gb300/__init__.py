"""GB300-native level-of-fill incomplete Cholesky IC(k) on the 2D partitioned-block
layout (Kim et al., arXiv:1601.05871): a C-ABI library (libick.so, include/ick.h)
with CUDA kernels for sm_103a and this thin Python binding.
"""
from .ick import (  # noqa: F401
    IckError,
    Handle,
    ic_nd_grid,
    ic_symbolic,
    ic_numeric,
    ic_apply,
    ic_apply_static,
    pcg_solve,
    ic_get_factor,
    ic_stats,
    ic_get_tasks,
    ic_block_dag,
    ic_get_task_targets,
    ic_get_upper,
    ic_get_blocks,
    ic_get_solve_tasks,
    ic_get_solve_trace,
    ic_get_solve_entries,
    ic_set_timing,
    ic_reset_timing,
    ic_get_timing,
    ic_test_hold_task,
    ic_set_trace,
    ic_get_trace,
    ic_destroy,
    load,
    IC_F64,
    IC_F32,
    TASK_NAMES,
)
from .ick import (  # noqa: F401,E402
    ic_symbolic_batch,
    ic_batch_info,
    pcg_solve_batch,
    ic_numeric_async,
    ic_numeric_status,
    ic_autotune,
)
