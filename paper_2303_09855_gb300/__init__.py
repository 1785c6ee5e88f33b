"""GB300-native IVF + ADSampling distance comparison operations.

The compute path is the C-ABI library ``libadsx.so`` (hand-written sm_103a
CUDA kernels, declared in ``include/adsx.h``); ``adsx`` is its thin Python
binding.  ``workloads`` makes seeded synthetic inputs.
"""
__all__ = ["adsx", "workloads"]
