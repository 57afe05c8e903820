"""GB300-native noisy surface-code state-vector trajectories (arXiv:2204.11404).

The simulation runs in libqecsv.so (hand-written CUDA for sm_103a behind the
C ABI of include/qecsv.h); ``capi`` is its ctypes binding.
"""
