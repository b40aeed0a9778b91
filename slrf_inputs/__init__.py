"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

Only input generation lives here (FEM pencil assembly, start blocks, workload
recipes); none of the eigensolver's arithmetic.
"""
from .fem import CsrPair, bar1d as bar1d_pencil, q1_elasticity, q1_scalar  # noqa: F401
from .configs import Workload, bar1d, q1_elast, q1_lap, start_block  # noqa: F401
