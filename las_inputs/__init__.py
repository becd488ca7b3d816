"""Seeded synthetic inputs shared by the oracle tests and the GPU library's tests and bench."""
from .gen import (BASE_SEED, WORKLOADS, LasSystem, batched_specs, batched_systems, make_system,
                  normals, npair, packed_B, packed_B_rows, splitmix64, uniforms,
                  workload_system)
from .rdm import fragment_rdms, nstrings, strings

__all__ = ["BASE_SEED", "WORKLOADS", "LasSystem", "batched_specs", "batched_systems",
           "workload_system", "make_system", "normals", "npair", "packed_B", "packed_B_rows",
           "splitmix64",
           "uniforms", "fragment_rdms", "nstrings", "strings"]
