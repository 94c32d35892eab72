"""GB300-native twisted-mass DD-alphaAMG (arXiv:1611.01034), Python binding.

A thin ctypes binding of the C ABI declared in ``include/tm.h``: the same
function names, argument marshalling only.  Every step of the solver runs in
the CUDA kernels of ``libtmamg.so``; there is no Python or CPU fallback, and
loading fails loudly if the library has not been built
(``python -m paper_1611_01034_gb300.build``).

Pointer arguments accept a torch tensor (its ``data_ptr()``), a numpy array
(host memory), a raw integer address or ``None`` (NULL).  Calls raise
:class:`TMError` on a non-zero status, except :func:`tm_solve`, which returns
``(status, info)`` so that a non-converged solve can still be inspected.
"""
from __future__ import annotations

import ctypes
import os

from ._binding import (  # noqa: F401
    TM_OK, TM_ERR_ARG, TM_ERR_CUDA, TM_ERR_OOM, TM_ERR_NOT_CONVERGED, TM_ERR_TIMEOUT,
    TM_ERR_NOT_SU3, TM_ERR_NONFINITE, TM_ERR_STATE, TM_F64, TM_F32, TM_F16, TM_BF16, TM_F32X2,
    TM_EXPORT_P, TM_EXPORT_DC, TM_EXPORT_CLOVER, TM_EXPORT_TV, TM_EXPORT_P2, TM_EXPORT_DC2, TM_EXPORT_TV1,
    TMError, tm_params, tm_solve_info, lib, library_path, params,
    tm_params_default, tm_create, tm_destroy, tm_status_string, tm_last_error,
    tm_load_gauge, tm_setup, tm_setup_from_vectors, tm_set_mu, tm_set_mu_eo, tm_autotune_build, tm_solve, tm_solve_squared, tm_solve_odd,
    tm_solve_hasenbusch,
    tm_solve_oecg,
    tm_field_bytes, tm_workspace_bytes, tm_save_setup, tm_load_setup, tm_pack, tm_unpack, tm_apply, tm_sap, tm_restrict, tm_prolong,
    tm_coarse_solve, tm_coarse_solve_noalloc, tm_kcycle, tm_setup_update, tm_schur, tm_nn_set_weights, tm_nn_get_weights, tm_nn_apply, tm_nn_pairs,
    tm_nn_grad, tm_nn_train, tm_sap1, tm_restrict1, tm_prolong1, tm_kcycle1,
    tm_export, tm_synchronize,
    tm_profile, tm_profile_kinds, tm_profile_name, tm_profile_read,
)
