"""GB300-native fluctuating D3Q19 lattice Boltzmann fluid with dissipative
point-particle coupling (variants A, B and C of Tretyakov & Duenweg,
arXiv:1610.02733), with the Kremer-Grest interactions of the paper's test
system.

The compute path lives in the CUDA library ``_build/liblbmd.so`` built from
``csrc/``; ``lbmd`` is its thin ctypes binding, ``inputs`` the seeded
synthetic-input generators, ``lj_units`` the conversion of the paper's
Lennard-Jones units and ``sweep`` the temperature-versus-friction experiment.
"""
