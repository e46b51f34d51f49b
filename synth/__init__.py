"""Seeded synthetic k-space inputs shaped like the HICU paper's workloads.

This package only makes data (phantoms, coil maps, sampling masks, noise).
It holds none of the reconstruction arithmetic, so both the FP64 oracle and
the CUDA path can consume its arrays without sharing any method code.
"""
from .phantoms import (  # noqa: F401
    Problem,
    centered_fft,
    make_problem,
    lowrank_exponential_kspace,
    CONFIG_NAMES,
)
