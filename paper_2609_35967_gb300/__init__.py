"""GB300-native collision step of GameDev's representative-particle Monte Carlo.

The hot path lives in libgd.so (hand-written CUDA for sm_103a behind the C ABI of
include/gd.h); `binding` is its thin ctypes binding and `workloads` the seeded
synthetic inputs.  Build with `python -m paper_2609_35967_gb300.build`.
"""
__all__ = ["binding", "workloads", "build"]
