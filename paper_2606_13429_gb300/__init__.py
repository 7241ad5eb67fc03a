"""GB300-native deflated conjugate gradient for the pseudo-stress Stokes system.

The compute path is libdcg.so (hand-written CUDA for sm_103a, C ABI in
include/dcg.h); `dcg` is its thin binding and `inputs` the seeded synthetic
input generator. Importing the package loads nothing; the library is loaded
on first use and raises if it is missing.
"""
