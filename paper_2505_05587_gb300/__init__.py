"""GB300 (sm_103a) implementation of the SteepGS splitting path.

libsteepgs.so (CUDA, include/steepgs.h) holds every kernel; ``binding`` is the
thin ctypes layer with the C names; ``pipeline`` owns buffers and orders the
calls of the fused fwd+bwd+splitting iteration.
"""
from . import binding  # noqa: F401
