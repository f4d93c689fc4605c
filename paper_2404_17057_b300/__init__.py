"""B300-native (sm_103a) hot path of the compressible-gas Material Point Method.

``mpm``     -- Python binding of the C ABI (include/mpm.h), libmpm.so
``inputs``  -- seeded synthetic initial conditions of the paper's test cases
``build``   -- compiles libmpm.so in-tree with nvcc for sm_103a
``serve``   -- continuous-batching request loop over many simulations
"""
