"""Seeded synthetic inputs for the response solver.

This module is shared by the CPU oracle tests and by the GPU path (tests,
``bench.py``, ``smoke()``).  It holds no arithmetic of the method itself: it
only draws atom positions, evaluates the external potential and the
perturbation as sums of periodic Gaussians on the real-space grid, and lists
Monkhorst-Pack k-points.  Every quantity the method computes (plane-wave
spheres, Fourier transforms, Hamiltonians, eigenpairs, occupations, densities,
kernels, responses) is computed separately by each side.
"""
from .systems import (System, make_system, perturbation, response_batch, loss_weights, CONFIGS,
                      TEST_SYSTEMS, monkhorst_pack, gaussian_sum_on_grid, supercell, with_kgrid,
                      with_cutoff)

__all__ = ["System", "make_system", "perturbation", "response_batch", "loss_weights", "CONFIGS",
           "TEST_SYSTEMS", "monkhorst_pack", "gaussian_sum_on_grid", "supercell", "with_kgrid",
           "with_cutoff"]
