"""GB300-native correlator X-engine (the hot path of arXiv 1503.06202).

For every frequency channel, the integrated visibility matrix
V_ij = sum_t x_i(t) conj(x_j(t)), i <= j, from 4+4-bit offset-encoded complex
voltages, computed exactly by hand-written sm_103a CUDA kernels behind the C
ABI in include/xeng.h.  ``xeng`` is the Python binding of that ABI.
"""
from .xeng import *  # noqa: F401,F403
from .xeng import XEngine, XengError, lib  # noqa: F401
