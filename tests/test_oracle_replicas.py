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
