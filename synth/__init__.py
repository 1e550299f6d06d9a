"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds no arithmetic of the method (no Dirac operator, no
solver, no force, no integrator).  It only draws random numbers from a
counter-based generator and shapes them into the fields the method
consumes: SU(3) link configurations, su(3) momenta, complex Gaussian
pseudofermion noise, sources and Metropolis uniforms.  Both the CPU oracle
and the CUDA path receive these arrays as inputs, so neither side draws
random numbers of its own.
"""
from .philox import philox4x32_10, uniform53, box_muller
from .fields import (Lattice, PRESETS, gauge_exp_iA, identity_gauge, momenta,
                     chi_noise, source, metropolis_uniform, gauge_transform,
                     plane_wave)

__all__ = ["philox4x32_10", "uniform53", "box_muller", "Lattice", "PRESETS",
           "gauge_exp_iA", "identity_gauge", "momenta", "chi_noise", "source",
           "metropolis_uniform", "gauge_transform", "plane_wave"]
