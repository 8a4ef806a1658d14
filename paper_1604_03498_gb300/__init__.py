"""GB300-native Fisher-vector encoder (GPU-FV, arXiv 1604.03498).

The encoder lives in a CUDA library with a C ABI (include/fv.h); the
``fv`` module is its thin Python binding and ``synth`` draws seeded
synthetic GMMs and descriptor sets.
"""
