"""Seeded synthetic survey generators shared by the oracle tests, the GPU tests and the bench.

This package holds inputs only: grids, velocity and reflectivity models, shot/receiver
geometry, frequency axes, the source wavelet spectrum and unit noise samples.  It contains
none of the migration arithmetic (no propagator, no operator, no solver), so both the FP64
oracle and the CUDA path can take their inputs from it without sharing any of the method.
"""

from .survey import (  # noqa: F401
    Survey,
    config_tiny,
    config_realistic,
    config_precision,
    config_midsize,
    config_precision_subsample,
    config_batching_lines,
    config_batching_lines_reduced,
    random_case,
    ricker_spectrum,
    linear_frequencies,
    centred_shots,
    full_spread_receivers,
    unit_complex_noise,
)
