"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle legs.

This package generates operands, moduli, lengths and job streams only.  It
holds none of the reduction arithmetic: it never computes an inverse, a
Montgomery constant or a reduction.  Both the library path and the oracle
consume what it produces.
"""

from .workloads import *  # noqa: F401,F403
