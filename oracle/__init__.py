"""FP64 CPU oracle for the StaRMAP staggered-grid P_N step.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py, never by the product path.
"""
from .pn_oracle import *  # noqa: F401,F403
