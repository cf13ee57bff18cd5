"""GB300 (sm_103a) two-lattice free energy lattice Boltzmann update.

A C-ABI CUDA library (``libfre.so``, declared in ``include/fre.h``) that
advances binary-mixture flows with the free energy LBM of Simonis et al.,
arXiv:2212.01617 (Sec. 2.2-2.3, Algorithm 1) on D2Q9 and D3Q19 lattices, in
the parallel-band shear and four-roller devices (Sec. 3), plus this thin
Python binding.  ``build.build()`` compiles the library in-tree.
"""
from .binding import (  # noqa: F401
    EXPORTS, FRE_BF16DEV, FRE_D2Q9, FRE_D3Q19, FRE_ERR_ARG, FRE_ERR_BUDGET, FRE_ERR_CUDA, FRE_ERR_OOM,
    FRE_ERR_STATE, FRE_ERR_UNSTABLE, FRE_FLAG_COUETTE_REFERENCE, FRE_FLAG_INTERPOLATED_WALLS,
    FRE_FLAG_REST_REFERENCE, FRE_FOUR_ROLLER, FRE_FP16DEV, FRE_FP32, FRE_FP64, FRE_OK, FRE_PERIODIC,
    FRE_SHEAR, Batch, FreError, Server, Simulation, fre_copy_fields, fre_create, fre_destroy, fre_device_bytes,
    fre_components, fre_init_droplet, fre_init_fields, fre_kernel_path, fre_last_error, fre_load_populations,
    fre_moments_noalloc, fre_observables, fre_params, fre_step, fre_step_count, fre_step_timed,
    fre_store_populations, fre_uses_row_kernels, load_library, make_params,
)

__all__ = [
    "EXPORTS", "FRE_BF16DEV", "FRE_D2Q9", "FRE_D3Q19", "FRE_ERR_ARG", "FRE_ERR_BUDGET", "FRE_ERR_CUDA",
    "FRE_ERR_OOM", "FRE_ERR_STATE", "FRE_ERR_UNSTABLE", "FRE_FLAG_COUETTE_REFERENCE", "FRE_FLAG_INTERPOLATED_WALLS",
    "FRE_FLAG_REST_REFERENCE", "FRE_FOUR_ROLLER", "FRE_FP16DEV", "FRE_FP32",
    "FRE_FP64", "FRE_OK", "FRE_PERIODIC", "FRE_SHEAR", "Batch", "FreError", "Server", "Simulation", "fre_copy_fields",
    "fre_components", "fre_create", "fre_destroy", "fre_device_bytes", "fre_init_droplet", "fre_init_fields", "fre_kernel_path",
    "fre_last_error", "fre_load_populations", "fre_moments_noalloc", "fre_observables", "fre_params",
    "fre_step", "fre_step_count", "fre_step_timed", "fre_store_populations", "fre_uses_row_kernels",
    "load_library", "make_params",
]
