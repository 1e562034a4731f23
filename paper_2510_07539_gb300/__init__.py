"""GB300-native semi-implicit IMEX step for the hyperbolic Serre-Green-Naghdi system.

The compute path is a CUDA library (``csrc/``, built for sm_103a) behind a C
ABI declared in ``include/hsgn.h``; ``solver`` is its thin Python binding.
``inputs`` holds the seeded synthetic workloads. Importing the package does not
load the CUDA library; ``solver`` does, and fails loudly if it is missing.
"""
__version__ = "0.1.0"
