"""Seeded synthetic workloads for the two-level block-Toeplitz MoM solver.

This package only draws inputs: basis centroids, generator blocks T[i,j],
excitation vectors and the uneven batch recipe.  It holds none of the
solver's arithmetic (no FFT, no product, no Krylov step), so both the CPU
oracle and the CUDA path may take their inputs from here.
"""
from .arrays import (  # noqa: F401
    ArraySpec,
    centroids,
    generator_blocks,
    periodic_generator_blocks,
    random_generator_blocks,
    port_index,
    port_excitations,
    centre_excitation,
    random_port_excitations,
    uneven_batch_specs,
    CONFIGS,
)
