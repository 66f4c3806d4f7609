"""GB300-native fluctuating D3Q19 lattice Boltzmann fluid with dissipative
point-particle coupling (variants A and B of Tretyakov & Duenweg,
arXiv:1610.02733).

The compute path lives in the CUDA library ``_build/liblbmd.so`` built from
``csrc/``; ``lbmd`` is its thin ctypes binding and ``inputs`` the seeded
synthetic-input generators.
"""
