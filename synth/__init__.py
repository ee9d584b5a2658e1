"""Seeded synthetic systems shared by the oracle tests and the GPU path.

This module only draws inputs (positions, charges, site maps, lambda values).
It contains none of the electrostatics or interpolation arithmetic."""
from .systems import CONFIGS, make, make_charges, make_e1, make_water, splitmix64, uniform01

__all__ = ["CONFIGS", "make", "make_charges", "make_e1", "make_water", "splitmix64", "uniform01"]
