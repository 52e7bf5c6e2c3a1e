"""B300-native isothermal MHD stepper (arXiv:2012.08758 hot path).

The compute path is the CUDA library ``libmhd_b300.so`` (hand-written
sm_103a kernels behind the C ABI of ``include/mhd.h``); this package is its
thin ctypes binding (same function names), a convenience ``Run`` wrapper
whose device workspace and stream come from PyTorch, the batch/serving
loop and the seeded input generators (``inputs``).

Importing the package is cheap; the library is loaded on first use and the
import of any binding name fails loudly if it is missing.
"""
from __future__ import annotations

_BINDING_NAMES = {
    "MhdError", "MhdParams", "lib", "mhd_default_params", "mhd_resolve_params", "mhd_workspace_bytes", "mhd_create",
    "mhd_destroy", "mhd_set_state", "mhd_get_state", "mhd_step", "mhd_step_timed", "mhd_reduce", "mhd_diagnostics",
    "mhd_time", "mhd_sync", "mhd_forcing_draw", "mhd_eval_rhs", "mhd_eval_rhs_at", "mhd_last_error",
    "mhd_batch_create", "mhd_batch_step", "mhd_batch_destroy", "MHD_F32", "MHD_F64",
    "REDUCE_NAMES", "MHD_URMS", "MHD_BRMS", "MHD_UMAX", "MHD_BMAX", "MHD_EKIN", "MHD_EMAG",
    "MHD_DIVB_MAX", "MHD_MASS", "MHD_VMAX", "MHD_NREDUCE", "MHD_KERNEL_AUTO", "MHD_KERNEL_SMEM",
    "MHD_KERNEL_TMA", "mhd_diagnostics_noalloc", "MHD_NOALLOC_MAX_POINTS", "mhd_alu_peak", "MHD_F32X2", "mhd_spectrum", "mhd_spectrum_shells", "mhd_set_seed_field", "mhd_substep_plan", "mhd_padding_check", "mhd_wait_selftest",
    "mhd_slabs_create", "mhd_slabs_extent", "mhd_slabs_set_state", "mhd_slabs_get_state", "mhd_slabs_step",
    "mhd_slabs_diagnostics", "mhd_slabs_destroy",
}


def __getattr__(name):
    if name in _BINDING_NAMES:
        from . import binding
        return getattr(binding, name)
    if name in ("Run", "Batch"):
        from . import run
        return getattr(run, name)
    if name == "Slabs":
        from . import slabs
        return slabs.Slabs
    raise AttributeError(name)
