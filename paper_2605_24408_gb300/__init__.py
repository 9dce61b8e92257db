"""GB300-native (sm_103a) p-dit probabilistic Ising machine for the symmetric QAP.

The product is the C-ABI library libpdit.so (include/pdit.h); `pdit` is its
Python binding, `instances` the seeded synthetic workload generator, `build`
the in-tree nvcc build.
"""

__all__ = ["pdit", "instances", "build"]
