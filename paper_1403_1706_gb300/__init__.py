"""GB300-native (sm_103a) filter-and-verify read mapping after Köster & Rahmann's PEANUT.

`peanut` is the Python binding of the C ABI in include/peanut.h (libpeanut.so, built by
`build.build()`).  All mapping work runs in the library's CUDA kernels.
"""
