"""CPU oracle for the market-split lattice method (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The CUDA product path never does.
"""
