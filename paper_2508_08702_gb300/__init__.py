"""GB300-native (sm_103a) lattice solver for the market split problem.

The package holds the CUDA sources (csrc/), their build script (build.py),
the Python binding of the C ABI (msp.py) and the seeded instance generators
(instances.py).  Importing the package loads nothing; ``msp.load()`` loads
the compiled library and fails loudly when it is missing.
"""

__all__ = ["build", "instances", "msp"]
