"""Pins for the general problem of Sec. 2 (bounds 0 <= x_j <= r_j): the
lattice of Eq. (2) with r_max = lcm(r) and c_j = r_max / r_j, the bounds
R = (n+1) r_max^2 and r_max ||w||_1 of the two pruning conditions, and the
generalised leaf test of Theorem 1.

The solution set has a plain definition -- every integer point of the box
with A x = d -- listed here by brute force over the box.  All-ones bounds
must reproduce the binary enumeration node for node."""
import numpy as np
import pytest

from oracle import definition as DEF
from oracle import oracle as O
from paper_2508_08702_gb300 import instances as I

MODES = [(O.HOELDER_CUT, True), (O.HOELDER_CUT, False), (O.HOELDER_FILTER, True), (O.HOELDER_OFF, True)]
CASES = [I.bounded(600 + s, m, n, D, bounds)
         for s in range(2)
         for (m, n, D, bounds) in [(1, 10, 30, (1, 2, 3)), (2, 12, 12, (1, 2, 3)), (2, 10, 20, (2, 4)),
                                   (3, 13, 8, (1, 3)), (2, 7, 25, (5, 7)), (2, 14, 6, (1, 2))]]


def test_lattice_columns():
    """Eq. (2): column 0 = (-N d, -r_max ..., r_max), column j = (N a_j, 2 c_j e_j, 0)."""
    A = np.array([[3, 5, 7]], np.int32)
    d = np.array([10], np.int64)
    r = np.array([2, 3, 4], np.int32)
    b = O.build_lattice(A, d, N=16, r=r)
    assert O.rmax(r) == 12
    assert b[0].tolist() == [-160, -12, -12, -12, 12]
    assert b[1].tolist() == [48, 12, 0, 0, 0]
    assert b[2].tolist() == [80, 0, 8, 0, 0]
    assert b[3].tolist() == [112, 0, 0, 6, 0]


@pytest.mark.parametrize("inst", CASES, ids=lambda x: x.tag)
@pytest.mark.parametrize("hoelder,sym", MODES)
def test_bounded_solution_sets_equal_brute_force(inst, hoelder, sym):
    want = DEF.brute_force_bounds(inst.A, inst.d, inst.r)
    assert any(np.array_equal(inst.planted, x) for x in want)
    got = O.solve(inst.A, inst.d, r=inst.r, hoelder=hoelder, sym=sym).result
    assert np.array_equal(got.solutions, want)


@pytest.mark.parametrize("seed", range(4))
def test_all_ones_bounds_are_the_binary_problem(seed):
    inst = I.small(1000 + seed, 3, 20, 8)
    ones = np.ones(inst.n, np.int32)
    a = O.solve(inst.A, inst.d).result
    b = O.solve(inst.A, inst.d, r=ones).result
    assert (a.nodes, a.passed, a.leaves) == (b.nodes, b.passed, b.leaves)
    assert np.array_equal(a.solutions, b.solutions)


def test_zero_slack_is_not_needed_to_be_sound_with_bounds():
    """The slack R 2^-20 only adds nodes: with and without it the bounded
    sets agree here (every solution sits on both bounds, as in the binary case,
    only when all c_j = 1; in general the check is the exact leaf test)."""
    inst = CASES[1]
    a = O.solve(inst.A, inst.d, r=inst.r).result
    b = O.solve(inst.A, inst.d, r=inst.r, use_eps=False).result
    assert set(map(bytes, b.solutions)) <= set(map(bytes, a.solutions))
    assert a.nodes >= b.nodes
