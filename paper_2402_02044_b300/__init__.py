"""LVQ search (arxiv 2402.02044) for NVIDIA B300 (sm_103a).

The compute lives in ``liblvq.so`` (hand-written CUDA behind the C ABI of
``include/lvq.h``); ``lvq`` is its ctypes binding and ``Store`` a small
owner of a store handle.  Import this package only where liblvq.so has been
built (``paper_2402_02044_b300.build.build()``).
"""
from .lvq import *  # noqa: F401,F403
from .lvq import Store, LVQError, load  # noqa: F401
