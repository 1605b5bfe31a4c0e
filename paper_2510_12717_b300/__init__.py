"""B300-native batched kinodynamic MPC (arXiv 2510.12717's GPU-parallel MPC hot path).

The compute path is the CUDA library libmpcgpu.so (C ABI, include/mpcgpu.h);
`mpcgpu` is its thin ctypes binding.  Importing this package does not load
the library; `paper_2510_12717_b300.mpcgpu.load()` does, and fails loudly when
it is missing.
"""
