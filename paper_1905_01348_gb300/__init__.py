"""GB300 library for parallel-transport Crank-Nicolson real-time TDDFT with a
screened hybrid functional (arXiv:1905.01348): the Fock exchange pair
pipeline, its ACE compression and the PT-CN step, as CUDA kernels behind the
C ABI of include/pt.h. This package is the thin Python binding.
"""
from ._native import (PT_FOCK_ACE, PT_FOCK_EXACT, PT_FOCK_NONE, PT_FP64, PT_MIXED, PtError, PtParams, PtStepInfo,
                      load, make_params, pt_apply_h, pt_basis_indices, pt_basis_size, pt_build_ace, pt_cn_step,
                      pt_destroy, pt_exchange, pt_get_orbitals, pt_init_system, pt_last_error, pt_observables,
                      pt_orbitals_device, pt_propagate, pt_set_orbitals, pt_workspace_size, pt_set_timing,
                      pt_get_timing, pt_launch_count, pt_exchange_static, pt_get_state, pt_set_state, pt_rk4_step,
                      pt_complex_product, pt_batch_workspace_size, pt_batch_create, pt_batch_exchange,
                      pt_batch_step, pt_batch_set_timing, pt_batch_get_timing, pt_batch_destroy, pt_seeded_coefficients)
from .system import Batch, System

__all__ = ["PT_FOCK_ACE", "PT_FOCK_EXACT", "PT_FOCK_NONE", "PT_FP64", "PT_MIXED", "PtError", "PtParams", "PtStepInfo",
           "System", "load", "make_params", "pt_apply_h", "pt_basis_indices", "pt_basis_size", "pt_build_ace",
           "pt_cn_step", "pt_destroy", "pt_exchange", "pt_get_orbitals", "pt_init_system", "pt_last_error",
           "pt_observables", "pt_orbitals_device", "pt_propagate", "pt_set_orbitals", "pt_workspace_size",
           "pt_set_timing", "pt_get_timing", "pt_launch_count", "pt_exchange_static", "pt_complex_product", "pt_get_state",
           "pt_set_state", "pt_rk4_step", "Batch", "pt_batch_workspace_size", "pt_batch_create", "pt_batch_exchange",
           "pt_batch_step", "pt_batch_set_timing", "pt_batch_get_timing", "pt_batch_destroy", "pt_seeded_coefficients"]
