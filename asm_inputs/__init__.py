"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package only builds matrices, partitions and right-hand sides; it holds
none of the preconditioner's arithmetic.
"""
from .rng import SplitMix64, mix64
from .problems import (Problem, poisson2d, diffusion3d, elasticity3d, convdiff2d,
                       stream_instance, config, contrast_field, rhs)

__all__ = ["SplitMix64", "mix64", "Problem", "poisson2d", "diffusion3d", "elasticity3d",
           "convdiff2d", "stream_instance", "config", "contrast_field", "rhs"]
