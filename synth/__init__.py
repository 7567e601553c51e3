"""Seeded synthetic workloads for the dust temperature / emission path.

This package only *makes inputs*: wavelength grids with their quadrature
weights, absorption cross sections of a toy grain model, heating fields and
grain number densities.  It holds none of the method's arithmetic (absorbed
power, temperature solve, emission) and is shared by the FP64 oracle, the CUDA
path, the tests and the benchmark, so that both sides see bit-identical inputs.
"""
from .workloads import (  # noqa: F401
    CONFIGS,
    SPECIES,
    Workload,
    blackbody_shape,
    cross_sections,
    fluctuating_selection,
    heat_capacity_params,
    grain_table,
    make_workload,
    wavelength_grid,
)
