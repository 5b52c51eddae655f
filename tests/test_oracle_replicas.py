"""Pins for the replicas' column orders (oracle/replicas.py)."""
import numpy as np

from oracle import definition as DEF
from oracle import oracle as O
from oracle import replicas as RP
from paper_2508_08702_gb300 import instances as I


def test_splitmix64_reference_output():
    """First output of splitmix64 from state 0, as published with the
    generator's reference implementation."""
    assert next(RP.splitmix64(0)) == 0xE220A8397B1DCDAF


def test_splitmix64_reference_sequence():
    """The first four outputs from state 0 of the published reference
    implementation."""
    g = RP.splitmix64(0)
    assert [next(g) for _ in range(4)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                           0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_fisher_yates_by_hand():
    """Replica 1 of instance 0 with seed 1 starts the stream at state
    1 ^ (0 << 32) ^ 1 = 0, so its z are the outputs above.  n = 4, from the
    identity (0, 1, 2, 3):
      j = 3: z1 mod 4 = 3 (last hex digit F = 15)        -> swap 3, 3: (0, 1, 2, 3)
      j = 2: z2 mod 3 = 0 (hex digit sum 135, 16 = 1 mod 3) -> swap 2, 0: (2, 1, 0, 3)
      j = 1: z3 mod 2 = 1 (last hex digit F, odd)          -> swap 1, 1: (2, 1, 0, 3)"""
    assert RP.permutation(4, 0, 1, seed=1).tolist() == [2, 1, 0, 3]


def test_permutations_are_permutations_and_differ():
    seen = set()
    for k in range(1, 6):
        p = RP.permutation(30, 2, k)
        assert sorted(p.tolist()) == list(range(30))
        seen.add(tuple(p.tolist()))
    assert len(seen) == 5
    assert RP.permutation(30, 2, 0).tolist() == list(range(30))


def test_shuffled_instance_has_the_permuted_solutions():
    inst = I.small(1001, 3, 20, 8)
    p = RP.permutation(inst.n, 0, 3)
    sols = O.solve(inst.A[:, p], inst.d).result.solutions
    back = np.zeros_like(sols)
    back[:, p] = sols
    assert np.array_equal(O.sort_solutions(back), DEF.brute_force(inst.A, inst.d))
