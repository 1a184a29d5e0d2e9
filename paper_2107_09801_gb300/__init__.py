"""GB300 library for the limited-neighbourhood search of Boskovic and Brest,
"Two-phase Optimization of Binary Sequences with Low Peak Sidelobe Level Value"
(arXiv 2107.09801).

Every step of the search runs in the CUDA kernels of ``libpsl.so``; this package
only marshals arguments to its C ABI (``include/psl.h``).  Importing it fails
loudly when the library has not been built: there is no CPU fallback.
"""
from .binding import (  # noqa: F401
    PSL_DONE, PSL_ERROR, PSL_FORM_BATCHED, PSL_FORM_PLAIN, PSL_QUEUED, PSL_RUNNING, TRACE_DTYPE, Context, PslError,
    lib_path, psl_autotune, psl_set_hot_config, psl_autocorr, psl_autocorr_static, psl_best, psl_config_default, psl_export_state, psl_init, psl_last_error, psl_poll,
    psl_profile, psl_profile_read, psl_release, psl_shutdown, psl_step, psl_submit, psl_submit_ex, psl_trace, psl_walk_bytes)
