"""Plain FP64 CPU oracle for the level-by-level multigrid Poisson solve on oct
grids (cuRAMSES, arXiv 2604.06035).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / reference legs.  The product package never
imports it, and it imports nothing from the product package.
"""
from .oracle import *  # noqa: F401,F403
