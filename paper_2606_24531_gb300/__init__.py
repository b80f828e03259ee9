"""GB300 (sm_103a) library for the two-layer codec of arXiv 2606.24531:
per-block interleaved-rANS entropy decode fused with absolute-offset LZ77
match resolution, for whole archives and for the unified single-coordinate
seek.  ``ace`` is the ctypes binding of the C ABI in include/ace.h;
``archive`` manages device memory for one archive with PyTorch.
"""
from . import ace  # noqa: F401
