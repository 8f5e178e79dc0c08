"""GB300-native Newton-step solver for the finite-strain multivariant
phase-field model of martensitic transformation (Tuma et al., CMAME 2021).

The computation lives in the CUDA library ``_lib/libpfm.so`` (C ABI in
include/pfm.h, sources in ``csrc/``); ``binding`` is its thin Python binding,
``inputs`` the seeded synthetic input generators, ``build`` the nvcc build.
Importing this package does not load the library; ``binding``/``abi`` raise
if it has not been built.
"""
__all__ = ["abi", "binding", "inputs", "build"]
