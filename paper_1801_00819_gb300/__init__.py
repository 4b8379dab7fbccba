"""GB300 (sm_103a) block-row recursive least-squares migration.

The compute path is liblsm_gb300.so (C ABI in include/lsm.h); ``lsm`` is its ctypes binding and
``device`` moves a synthetic survey into the argument holders and device tensors the binding
takes.  Build the library with ``python -m paper_1801_00819_gb300.build``.
"""

from .lsm import (  # noqa: F401
    Frequencies,
    Geometry,
    Grid,
    LineProblem,
    LsmError,
    lsm_adjoint,
    lsm_autotune,
    lsm_autotune_reset,
    lsm_autotune_gradient,
    lsm_born_gradient,
    lsm_fft_tiles,
    lsm_forward,
    lsm_kernel_launches,
    lsm_measure_fp32_peak,
    lsm_num_windows,
    lsm_profile_start,
    lsm_profile_stop,
    lsm_status_string,
    lsm_workspace_bytes,
    rls_multi_line_solve,
    rls_window_solve,
    LSM_OP_FORWARD,
    LSM_OP_ADJOINT,
    LSM_OP_SOLVE,
    LSM_OP_GRADIENT,
)
