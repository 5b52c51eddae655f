"""Column orders of the replica portfolio (test infrastructure only).

Sec. 4 suggests running the method on several randomly shuffled input
orders at once.  The library shuffles replica k > 0 of instance i on the
device; this module restates the same published generators independently so
that tests can rebuild each replica on the CPU:

* splitmix64 (Steele, Lea and Flood, 2014): state += 0x9E3779B97F4A7C15,
  z = state; z = (z ^ z >> 30) * 0xBF58476D1CE4E5B9;
  z = (z ^ z >> 27) * 0x94D049BB133111EB; output z ^ z >> 31 (mod 2^64);
* Fisher-Yates: for j = n-1 down to 1, swap positions j and z mod (j+1),
  z the next splitmix64 output, starting from the identity;
* the stream of replica k of instance i starts at seed ^ (i << 32) ^ k.

perm[j] is the original column that becomes column j of the replica.
"""
from __future__ import annotations

import numpy as np

MASK = (1 << 64) - 1
DEFAULT_SEED = 0x5EED5EED5EED5EED


def splitmix64(state: int):
    """Generator of splitmix64 outputs from the given state."""
    while True:
        state = (state + 0x9E3779B97F4A7C15) & MASK
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        yield z ^ (z >> 31)


def permutation(n: int, instance: int, replica: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    perm = list(range(n))
    if replica == 0:
        return np.array(perm, dtype=np.int64)
    gen = splitmix64((seed ^ (instance << 32) ^ replica) & MASK)
    for j in range(n - 1, 0, -1):
        k = next(gen) % (j + 1)
        perm[j], perm[k] = perm[k], perm[j]
    return np.array(perm, dtype=np.int64)
