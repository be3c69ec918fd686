"""GB300-native inexact policy iteration for finite discounted MDPs.

``build`` compiles the CUDA library (libmdp.so, C ABI in include/mdp.h) and
``mdp`` is its Python binding.  Nothing here computes on the CPU.
"""
