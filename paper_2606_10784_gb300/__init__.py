"""GB300-native numerically filtered Adaptive Integral Method (2-D EFIE).

The compute path lives in the CUDA library `libaimgb300.so` (C ABI in include/aim.h);
`paper_2606_10784_gb300.aim` is its ctypes binding. Importing the package does not load the
library; `aim.lib()` does, and raises if it has not been built.
"""
