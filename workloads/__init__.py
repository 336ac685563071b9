"""Seeded synthetic inputs shared by the FP64 oracle and the GPU path.

Holds circuit descriptions only (gate names, qubits, angles, random draws);
no simulation arithmetic lives here.
"""
from .circuits import *  # noqa: F401,F403
from .circuits import GATES, Op, Circuit  # noqa: F401
