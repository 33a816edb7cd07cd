"""GB300-native Segment Linking (Line Segment Tracking, arXiv:2209.13711).

The chain runs in the CUDA kernels of liblst.so (csrc/, C ABI in
include/lst.h); `lst` is the thin Python binding. Around it: `serve` (a
serving loop with continuous batching), `train` (the T5 scoring network on
the device), `metrics` (efficiency, fake and duplicate rates on generator
truth) and `run` (a command-line driver).
"""
from .lst import (Context, LstError, Mlp, TC_DTYPE, default_capacity, default_config, library,  # noqa: F401
                  build_mini_doublets_static, measure_peaks, pack_events, tc_dict)
