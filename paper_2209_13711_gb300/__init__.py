"""GB300-native Segment Linking (Line Segment Tracking, arXiv:2209.13711).

The chain runs in the CUDA kernels of liblst.so (csrc/, C ABI in
include/lst.h); `lst` is the thin Python binding.
"""
from .lst import Context, LstError, Mlp, default_capacity, default_config, library, pack_events  # noqa: F401
