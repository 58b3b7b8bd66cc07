"""GB300-native ARP-blocked ALIF simulation (Taylor, King & Harper, NeurIPS 2023).

The compute path lives in the CUDA library built from `csrc/` (C ABI declared in
include/alif.h); `alif` is its thin ctypes binding.  `synth` holds the seeded
synthetic workloads.
"""
