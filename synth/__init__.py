"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package draws random wire clouds, incidence lists and observation lists. It holds
none of the method's arithmetic: no Green's function, no quadrature, no solver.
"""
from .clouds import (  # noqa: F401
    Cloud,
    cloud_small,
    cloud_mid,
    cloud_batching_snapshot,
    batching_sizes,
    cloud_precision,
    cloud_learned,
    cloud_uniform_cube,
    cloud_single,
    cloud_by_name,
    incidences_single_minus_z,
    incidences_monostatic,
    observations_phi_cut,
    CONFIGS,
)
