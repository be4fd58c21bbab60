"""GB300-native brute-force incoherent de-dispersion (ARTEMIS, Sec. 2-3).

The compute path is libdd.so (hand-written sm_103a CUDA behind a C ABI, see
include/dd.h); this package is its thin Python binding.  Importing it loads
the library and raises ImportError if it has not been built
(``python __graft_entry__.py``).
"""
from ._binding import (DD_F16, DD_F32, DD_U8, Batch, add_peak, DDError, Plan, Server, Tiles, channelise,
                       channelise_nspec, check, detect, dtype_code, elem_size, frontend,
                       frontend_work_bytes, launch_count, lib, pfb_prototype, profile_events,
                       unpack, warp_span)

__all__ = ["Plan", "Batch", "Server", "Tiles", "DDError", "DD_U8", "DD_F16", "DD_F32", "check",
           "dtype_code", "elem_size", "warp_span", "launch_count", "profile_events", "unpack",
           "detect", "frontend", "frontend_work_bytes", "channelise", "channelise_nspec",
           "pfb_prototype", "lib", "add_peak"]
