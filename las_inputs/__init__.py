"""Seeded synthetic inputs shared by the oracle tests and the GPU library's tests and bench."""
from .gen import (BASE_SEED, CONFIGS, LasSystem, batched_specs, batched_systems, config_system,
                  make_system, normals, npair, packed_B, packed_B_rows, splitmix64,
                  uniforms)
from .rdm import fragment_rdms, nstrings, strings

__all__ = ["BASE_SEED", "CONFIGS", "LasSystem", "batched_specs", "batched_systems",
           "config_system", "make_system", "normals", "npair", "packed_B", "packed_B_rows",
           "splitmix64",
           "uniforms", "fragment_rdms", "nstrings", "strings"]
