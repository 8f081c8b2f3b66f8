"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds only random-number generation and the bunch recipes of
the workloads (distribution shapes and sizes). It holds none of the
tracking, network or moment arithmetic of the method, so both sides can
consume the same arrays without sharing any of that code.
"""
from .philox import philox4x32_10, uniform53, normal_pairs
from .bunch import (BunchRecipe, ELECTRON_REST_MEV, gamma_from_kinetic_gev,
                    gaussian_bunch, training_population, uneven_counts,
                    random_quad_magnitudes, mlp_init)

__all__ = [
    "philox4x32_10", "uniform53", "normal_pairs", "BunchRecipe",
    "ELECTRON_REST_MEV", "gamma_from_kinetic_gev", "gaussian_bunch",
    "training_population", "uneven_counts", "random_quad_magnitudes",
    "mlp_init",
]
