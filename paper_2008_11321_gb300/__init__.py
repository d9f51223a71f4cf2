"""GB300-native (sm_103a) ADG + JP-ADG graph colouring.

The computation lives in ``libgcolor.so`` (CUDA kernels behind the C ABI of
include/gcolor.h); ``gcolor`` is its thin ctypes binding.  Importing the
package does not load the library: the first call does, and fails loudly if
it is missing.
"""
from .gcolor import (Context, DeviceBatch, DeviceGraph, GcError, GC_ERR_CUDA, GC_ERR_INVALID_ARG,  # noqa: F401
                     GC_ERR_INVALID_GRAPH, GC_ERR_OOM, GC_ERR_OVERFLOW, GC_ERR_TIMEOUT, GC_OK,
                     GC_PRIO_FF, GC_PRIO_LF, GC_PRIO_LLF, GC_PRIO_R, GC_PRIO_SL, GC_UPDATE_AUTO, GC_UPDATE_PULL, GC_BATCH_AUTO,
                     GC_BATCH_PERSISTENT, GC_BATCH_SEGMENTED,
                     GC_UPDATE_PUSH, EXPORTS, LIB_PATH, gc_options, load, make_options, status_str)

__all__ = ["Context", "DeviceBatch", "DeviceGraph", "GcError", "load", "make_options", "gc_options", "status_str",
           "EXPORTS", "LIB_PATH"]
