"""GB300 (sm_103a) Dynamic Frontier PageRank (arXiv 2401.03256).

The compute lives in libprdf.so (CUDA, C ABI in include/prdf.h); ``prdf`` is its ctypes
binding and ``build`` compiles it in-tree.
"""
from . import build  # noqa: F401
