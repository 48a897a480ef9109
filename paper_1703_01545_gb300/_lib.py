"""ctypes view of include/afqmc.h: struct layouts and function signatures.

Loading fails loudly when the shared library is missing; there is no fallback.
"""
import ctypes
import os

from .build import LIB

c_double_p = ctypes.POINTER(ctypes.c_double)


class AfqmcOptions(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("n_walkers", ctypes.c_int),
                ("taylor_order", ctypes.c_int), ("precision", ctypes.c_int),
                ("mode", ctypes.c_int), ("n_repeats", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("fb_cap", ctypes.c_double),
                ("walker_offset", ctypes.c_int64), ("autotune", ctypes.c_int),
                ("autotune_cache", ctypes.c_char_p), ("independent_fields", ctypes.c_int)]


class AfqmcInfo(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("X", ctypes.c_int), ("n_up", ctypes.c_int),
                ("n_dn", ctypes.c_int), ("n_walkers", ctypes.c_int), ("n_repeats", ctypes.c_int),
                ("step", ctypes.c_uint64), ("e_trial", ctypes.c_double),
                ("c_mf", ctypes.c_double), ("n_alive", ctypes.c_int),
                ("tuned_energy_walkers_per_cta", ctypes.c_int), ("tuned_taylor_smem", ctypes.c_int),
                ("tuned_orthonormalise", ctypes.c_int), ("n_det", ctypes.c_int)]


STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "numerical failure",
          4: "invalid state", 5: "device wait timed out", 6: "out of device memory"}

# name -> (restype, argtypes); every symbol include/afqmc.h declares
VP = ctypes.c_void_p
SIGNATURES = {
    "afqmc_default_options": (None, [ctypes.POINTER(AfqmcOptions)]),
    "afqmc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "afqmc_last_error": (ctypes.c_char_p, [VP]),
    "afqmc_setup": (ctypes.c_int, [ctypes.POINTER(VP), VP, VP, VP, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, ctypes.POINTER(AfqmcOptions), VP]),
    "afqmc_setup_multidet": (ctypes.c_int, [ctypes.POINTER(VP), VP, VP, VP, VP, ctypes.c_int, VP,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(AfqmcOptions), VP]),
    "afqmc_destroy": (ctypes.c_int, [VP]),
    "afqmc_set_walkers": (ctypes.c_int, [VP, VP, VP, VP]),
    "afqmc_get_state": (ctypes.c_int, [VP, VP, VP, VP, VP, VP]),
    "afqmc_set_step": (ctypes.c_int, [VP, ctypes.c_uint64, VP]),
    "afqmc_population_control": (ctypes.c_int, [VP, VP, VP]),
    "afqmc_seed_secondary": (ctypes.c_int, [VP, VP, VP]),
    "afqmc_get_info": (ctypes.c_int, [VP, ctypes.POINTER(AfqmcInfo), VP]),
    "afqmc_propagate": (ctypes.c_int, [VP, ctypes.c_int, VP, VP]),
    "afqmc_orthonormalise": (ctypes.c_int, [VP, VP]),
    "afqmc_energy": (ctypes.c_int, [VP, VP, VP, VP, VP]),
    "afqmc_pair_delta_E": (ctypes.c_int, [VP, VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, VP, VP, VP, VP, VP]),
    "afqmc_pair_graph_kernels": (ctypes.c_int, [VP, ctypes.POINTER(ctypes.c_int)]),
    "afqmc_pair_run_form": (ctypes.c_int, [VP, ctypes.POINTER(ctypes.c_int)]),
    "afqmc_delta_E_stats": (ctypes.c_int, [VP, VP, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           VP, VP, VP]),
    "afqmc_reblock_error": (ctypes.c_double, [VP, ctypes.c_int]),
    "afqmc_set_tangent": (ctypes.c_int, [VP, VP, VP]),
    "afqmc_energy_tangent": (ctypes.c_int, [VP, VP, VP, VP, VP]),
    "afqmc_get_tangent_state": (ctypes.c_int, [VP, VP, VP]),
    "afqmc_select_kernel": (ctypes.c_int, [VP, ctypes.c_int, ctypes.c_int]),
    "afqmc_adjoint_run": (ctypes.c_int, [VP, ctypes.c_int, VP, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, VP, VP, VP]),
    "afqmc_local_energy_static": (ctypes.c_int, [VP, VP, VP, VP, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_int, ctypes.c_int, VP,
                                                 VP]),
    "afqmc_test_gemm": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, VP,
                                       VP, ctypes.c_double, VP, VP]),
    "afqmc_time_kernel": (ctypes.c_int, [VP, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_double), VP]),
}

_lib = None


def load(path: str = LIB):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: the AFQMC CUDA library must be built first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
