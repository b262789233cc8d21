"""GB300-native Blind-Match: encrypted 1:N cosine-similarity matching under RNS-CKKS.

The compute path lives in the CUDA library `libblindmatch.so` (sources in
`csrc/`, C-ABI declared in `include/blindmatch.h`); `binding` is its thin
ctypes wrapper and `workload` the seeded synthetic-feature generator.
"""
