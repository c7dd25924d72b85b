"""Plain FP64 CPU oracle of the split pressure-gradient projection.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference legs may import anything from here.  The CUDA product
path never imports, calls or links this package, and this package imports
nothing from the product package.
"""
from .ppe_oracle import *  # noqa: F401,F403
