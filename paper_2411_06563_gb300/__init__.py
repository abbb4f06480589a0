"""GB300-native implementation of the HOSC scheme for 3D power-law natural convection.

The compute path is libhosc.so (CUDA, sm_103a) behind the C ABI of include/hosc.h; ``hosc`` is its
Python binding and ``inputs`` holds seeded synthetic input generators.
"""

__all__ = ["hosc", "inputs", "build"]
