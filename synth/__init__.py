"""Seeded synthetic inputs (scenes, cameras) for the 3DGS training hot path.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic.  Both the FP64 oracle and the CUDA path take their inputs
from here.
"""
from .scenes import *  # noqa: F401,F403
