"""GB300-native (sm_103a) Louvain community detection: local-moving and aggregation on the GPU.

The compute path is the CUDA library ``libgblouvain.so`` behind the C ABI in
``include/louvain.h``; :mod:`.louvain` binds it with ctypes.  Build it with
:func:`paper_2301_12390_gb300.build.build`.
"""
from .louvain import (ASYNC, PTR_DEVICE, PTR_HOST, SYNC, Louvain, LouvainError, Options, Server, arena_bytes,
                      default_options, load_library)

__all__ = ["Louvain", "LouvainError", "Options", "Server", "arena_bytes", "default_options", "load_library", "SYNC",
           "ASYNC", "PTR_HOST", "PTR_DEVICE"]
