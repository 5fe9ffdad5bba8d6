"""GB300 node-aware parallel SpMV (NAPSpMV, Bienz, Gropp, Olson, arXiv 1612.08060).

The compute path is libnapspmv.so (hand-written sm_103a CUDA behind the C ABI of
include/napspmv.h); ``napspmv`` is its thin Python binding, ``inputs`` the seeded
synthetic workloads, ``serve`` the continuous-batching request server and
``autotune`` the launch-option tuner.
"""
