"""GB300 (sm_103a) library for the density-fitted LAS energy and orbital gradient.

The compute lives in liblasdf.so (C ABI declared in include/las.h); this package is its thin
Python binding.  There is no CPU fallback.
"""
from .las import (EXPORTS, LAS_FP64, LAS_SPLIT_BF16, LasDF, LasError, aux_range,
                  aux_shard_partial, energy_grad_aux_sharded, energy_grad_batched, kernel_launches, las_energy,
                  load_library, probe_fp64, selftest_bounded_wait, split_gemm)

__all__ = ["EXPORTS", "LAS_FP64", "LAS_SPLIT_BF16", "LasDF", "LasError", "las_energy",
           "load_library", "kernel_launches",
           "split_gemm", "energy_grad_batched", "selftest_bounded_wait", "aux_range",
           "aux_shard_partial", "energy_grad_aux_sharded", "probe_fp64"]
