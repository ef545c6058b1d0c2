"""FP64 CPU oracle for the semi-coherent track statistic (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline may import
this package; the product path never does.
"""
from .tfstat_oracle import *  # noqa: F401,F403
