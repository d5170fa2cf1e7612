"""GB300-native Hough-transform track finding (arXiv:1309.6275, Sections 5-7).

The hot path -- vote, peak finding, hit association and the (z0, cot theta)
vote -- runs in libht's hand-written CUDA kernels for sm_103a behind the C ABI
of include/ht.h.  ``paper_1309_6275_gb300.ht`` is its thin Python binding.
"""
from . import build

__all__ = ["build"]
