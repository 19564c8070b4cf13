"""Seeded synthetic speckle bursts (test and benchmark input only).

This package simulates the data a speckle camera records: a granulation-like
scene, Kolmogorov seeing over a circular pupil, detector noise and 12-bit
quantisation.  It holds no step of the reconstruction itself, so both the
CUDA path and the FP64 oracle can take their inputs from it.
"""
from .burst import (  # noqa: F401
    BurstSpec,
    CONFIGS,
    make_burst,
    make_object,
    kolmogorov_psf,
    diffraction_psf,
    empirical_stf,
)
