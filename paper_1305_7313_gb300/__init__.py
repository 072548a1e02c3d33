"""GB300 Fock exact-exchange operator (arXiv:1305.7313, §4).

The C ABI of ``libfockx.so`` (include/fock.h) is exposed under the same names in
``paper_1305_7313_gb300._lib``; this module adds a small object wrapper,
:class:`FockPlan`, whose methods call those entry points.  Every step of the
computation runs in the library's CUDA kernels; PyTorch provides device memory
and streams only.  The library is loaded on first use and a missing build
raises immediately.
"""

from ._lib import (  # noqa: F401
    ERFC,
    GAMMA_REAL,
    PREC_DF64,
    PREC_FP64,
    PREC_MIXED32,
    SPENCER_ALAVI,
    FockError,
    fock_apply,
    fock_apply_fixed,
    fock_set_occupied,
    fock_batch_create,
    fock_batch_default_options,
    fock_batch_destroy,
    fock_batch_info,
    fock_batch_last_error,
    fock_batch_run,
    fock_apply_shard,
    fock_destroy,
    fock_gsphere,
    fock_kplan_apply,
    fock_kplan_create,
    fock_kplan_destroy,
    fock_kplan_gvectors,
    fock_kplan_set_batch,
    fock_last_error,
    fock_pair_energies,
    fock_pair_energies_static,
    fock_schedule,
    fock_plan_create,
    fock_plan_columns,
    fock_plan_set_deterministic,
    fock_plan_device_bytes,
    fock_plan_gvectors,
    fock_plan_npw,
    fock_plan_reserve,
    fock_plan_set_band_block,
    fock_plan_set_batch,
    fock_plan_set_streams,
    fock_plan_set_tiling,
    fock_plan_set_timing,
    fock_plan_stats,
    fock_plan_tiling_info,
    fock_status_string,
)
from .plan import FockBatch, FockKPlan, FockPlan  # noqa: F401
