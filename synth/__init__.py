"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This package draws orbital energies and density-fitting factors.  It holds
none of the EA-ADC arithmetic: it only produces the inputs both sides
consume, so that the two compute on bit-identical data.
"""
from .generator import (  # noqa: F401
    splitmix64, uniform53, normal01, make_problem, CONFIGS, config_problem,
)
