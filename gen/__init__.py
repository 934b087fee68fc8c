"""Seeded synthetic particle clouds shaped like the paper's GMC workloads.

This package holds input generation only (positions, masses, softening radii,
sink flags, active subsets, cotangents). It contains none of the gravity
method's arithmetic, and both the CUDA path's tests/bench and the CPU oracle
draw their inputs from it.
"""
from .clouds import (Cloud, uniform_cloud, clumpy_cloud, adjoint_cloud, ensemble,
                     paper_scale_cloud, active_subset, cotangents, CONFIG_SEED)

__all__ = ["Cloud", "uniform_cloud", "clumpy_cloud", "adjoint_cloud", "ensemble",
           "paper_scale_cloud", "active_subset", "cotangents", "CONFIG_SEED"]
