"""GB300 (sm_103a) QG beta-plane LES step behind the libqg C-ABI.

Python names mirror include/qg.h; the functions only marshal arguments and
every step of the computation runs in libqg's CUDA kernels.
"""
from ._lib import (QG_DLEITH, QG_DSMAG, QG_ERR_ARG, QG_ERR_BOUNDS, QG_ERR_CUDA, QG_ERR_NONFINITE, QG_ERR_OOM,
                   QG_ERR_TIMEOUT, QG_ERR_UNSUPPORTED,
                   QG_FP32, QG_FP64, QG_LEITH, QG_NONE, QG_OK, QG_SCHEME_AB2CN, QG_SCHEME_RK3_EXACT, QG_SMAG,
                   QGError, load)
from .qg import (QGEnsemble, QGSolver, qg_create, qg_destroy, qg_diagnostics, qg_get_state, qg_grid_filter, qg_last_error,
                 qg_series_compare, qg_set_state, qg_sgs_apriori, qg_step, qg_step_vjp, qg_stream, qg_sync, qg_version)

__all__ = [
    "QGSolver", "QGEnsemble", "QGError", "load", "qg_create", "qg_destroy", "qg_diagnostics", "qg_get_state", "qg_set_state",
    "qg_sgs_apriori", "qg_grid_filter", "qg_series_compare", "qg_step_vjp", "qg_step", "qg_stream", "qg_sync", "qg_last_error", "qg_version",
    "QG_NONE", "QG_SMAG", "QG_LEITH", "QG_DSMAG", "QG_DLEITH", "QG_FP32", "QG_FP64",
    "QG_SCHEME_RK3_EXACT", "QG_SCHEME_AB2CN",
    "QG_OK", "QG_ERR_ARG", "QG_ERR_CUDA", "QG_ERR_NONFINITE", "QG_ERR_OOM", "QG_ERR_UNSUPPORTED", "QG_ERR_TIMEOUT",
    "QG_ERR_BOUNDS",
]
