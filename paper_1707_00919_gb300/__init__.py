"""GB300 (sm_103a) parallel multicanonical simulation of the 2D Ising model
(Gross, Zierenberg, Weigel, Janke, arXiv:1707.00919).

The product is libmuca.so (C ABI in include/muca.h); this package holds its CUDA/C++
sources (csrc/), the in-tree build (build.py) and the Python binding (muca.py).
"""
from .muca import (MUCA_LAYOUT_AUTO, MUCA_LAYOUT_INT8, MUCA_LAYOUT_PACKED, MUCA_SCHEDULE_PAPER,  # noqa: F401
                   MUCA_WPB_TUNE,
                   MUCA_SCHEDULE_SWEEPS, MUCA_STOP_CHEBYSHEV, MUCA_STOP_KL, MUCA_STOP_MIN_MEAN,
                   Batch, IterationStats, Muca, MucaError, Server, make_params)
