"""GB300-native correlated-sampling phaseless AFQMC walker propagation.

The compute lives in the sm_103a CUDA library ``libafqmc_gb300.so`` (C ABI in
include/afqmc.h); this package is its build script and ctypes binding.
"""
from .api import (BF16X3, FP64, FREE, PHASELESS, AfqmcError, System, afqmc_default_options,
                  afqmc_delta_E_stats, afqmc_destroy, afqmc_energy, afqmc_get_info,
                  afqmc_get_state, afqmc_orthonormalise, afqmc_pair_delta_E,
                  afqmc_pair_graph_kernels, afqmc_pair_run_form, afqmc_propagate, afqmc_reblock_error,
                  afqmc_set_step, afqmc_set_walkers, afqmc_setup, afqmc_setup_multidet,
                  afqmc_time_kernel, pair_delta_E,
                  afqmc_population_control, afqmc_seed_secondary,
                  pair_graph_kernels, pair_run_form, K_VHS, K_FORCE_BIAS, K_TAYLOR, K_EXCHANGE,
                  K_OVERLAP, K_OVERLAP_UPDATE, K_MGS, K_PAIR_LOOP)
from .build import build

__all__ = ["System", "pair_delta_E", "pair_graph_kernels", "pair_run_form", "build", "AfqmcError", "PHASELESS", "FREE", "FP64", "BF16X3",
           "afqmc_default_options", "afqmc_setup", "afqmc_setup_multidet", "afqmc_destroy", "afqmc_set_walkers", "afqmc_set_step",
           "afqmc_population_control", "afqmc_seed_secondary",
           "afqmc_get_state", "afqmc_get_info", "afqmc_propagate", "afqmc_orthonormalise",
           "afqmc_energy", "afqmc_pair_delta_E", "afqmc_pair_graph_kernels", "afqmc_pair_run_form", "afqmc_delta_E_stats", "afqmc_reblock_error",
           "afqmc_time_kernel", "K_VHS", "K_FORCE_BIAS", "K_TAYLOR", "K_EXCHANGE", "K_OVERLAP",
           "K_OVERLAP_UPDATE", "K_MGS", "K_PAIR_LOOP"]
