"""Seeded synthetic inputs for the JAGP VMC hot path.

This module only *draws* inputs (atom positions, basis exponents, the pairing
matrix lambda, Jastrow parameters, initial walker positions).  It holds none of
the method's arithmetic, so both the CPU oracle and the CUDA library can take
their inputs from it without sharing any computation.
"""
from .systems import (  # noqa: F401
    System,
    config1,
    config2,
    config3_systems,
    config4,
    config5,
    hydrogen_slater,
    hydrogenic_gauss_j1,
    one_electron_slater,
    one_electron_gauss,
    helium_slater,
    small_random,
    with_j3,
    init_walkers,
    jitter_walkers,
    CONFIGS,
)
