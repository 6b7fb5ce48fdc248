"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

Holds geometry and random inputs only, none of the method's arithmetic.
"""
from .lattice import Cluster, honeycomb, named, relabel, translations, characters, GAMMA_X, GAMMA_Y, GAMMA_Z  # noqa: F401
from .states import random_state, random_vectors, hashed_amplitudes, omega_grid, log_temperatures  # noqa: F401
