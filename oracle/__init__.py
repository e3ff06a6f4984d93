"""FP64 CPU oracle of the QMCUR hot path (arXiv 2402.19147).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU legs of bench.py; never by the library.  It is independent of the CUDA
path (no shared code, no shared constants, neither imports the other).
"""
from . import quat, philox, qmcur  # noqa: F401
