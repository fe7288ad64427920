"""GB300-native Jacobi-PCG for the linear finite-difference Poisson-Boltzmann equation.

The compute path lives in ``libpb.so`` (hand-written CUDA for sm_103a behind a
C ABI, sources in ``csrc/``); ``pb`` is its thin ctypes binding and
``inputs`` holds the seeded synthetic workload generators.
"""
