"""Exact Density-Peaks Clustering on one NVIDIA GB300 (sm_103a).

Python binding of ``libdpc`` (C ABI declared in ``include/dpc.h``). Every
step of the clustering runs in the library's CUDA kernels; this package only
marshals arguments (numpy arrays, torch tensors, pointers, streams). There is
no CPU fallback: if the library cannot be built or loaded, importing the
binding's entry points raises.

Low-level functions carry the C names (``dpc_create``, ``dpc_density``,
``dpc_dependent``, ``dpc_label``, ``dpc_release``, ``dpc_submit``,
``dpc_poll``, ``dpc_flush``, ``dpc_wait``, ...). ``Context`` / ``Dataset``
wrap them, and ``cluster()`` runs the whole path on host arrays
(``cluster_approx()`` and ``cluster_sapprox()`` the approximate ones).
"""
from ._binding import (  # noqa: F401
    DPC_OK, DPC_PENDING, DPC_ERR_INVALID_ARG, DPC_ERR_OOM, DPC_ERR_CUDA, DPC_ERR_TIMEOUT,
    DPC_ERR_STATE, DPC_ERR_CAPACITY, INT64_MAX, DpcError, Context, Dataset, Job, cluster, cluster_approx, cluster_sapprox, lib,
    dpc_create, dpc_destroy, dpc_density, dpc_dependent, dpc_label, dpc_release, dpc_ds_info,
    dpc_last_batch_info, dpc_autotune, dpc_dependent_approx, dpc_sapprox, dpc_cluster, eps_fraction,
    dpc_set_profiling, dpc_submit, dpc_poll, dpc_flush, dpc_wait, dpc_last_error, library_path,
    dpc_kernel_launches, dpc_probe_pair_rate, dpc_set_tuning, dpc_get_tuning, dpc_job_footprint,
)
