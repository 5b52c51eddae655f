"""Pins for the oracle's enumeration (Algorithm 1, Theorems 1 and 2).

The solution set has a plain definition -- {x in {0,1}^n : A x = d} -- so the
enumeration oracle is pinned against brute force and meet-in-the-middle
(oracle/definition.py), across every pruning mode, on instances chosen to
have many solutions (small D), so that a wrong sign, index or dropped term in
the centre, the norms, the zig-zag or the direction cut loses solutions.
"""
import numpy as np
import pytest

from oracle import definition as DEF
from oracle import oracle as O
from paper_2508_08702_gb300 import instances as I

MODES = [(O.HOELDER_CUT, True), (O.HOELDER_CUT, False), (O.HOELDER_FILTER, True),
         (O.HOELDER_FILTER, False), (O.HOELDER_OFF, True), (O.HOELDER_OFF, False)]

SMALL = [I.small(1000 + s, m, n, D)
         for s in range(6)
         for (m, n, D) in [(1, 16, 60), (2, 18, 12), (3, 20, 8), (2, 20, 30), (4, 22, 6),
                           (3, 21, 100)]]


def test_definition_hand_example():
    """A = [1 2 3], d = 3: x = (1,1,0) and (0,0,1), checked by hand."""
    A = np.array([[1, 2, 3]])
    d = np.array([3])
    want = np.array([[0, 0, 1], [1, 1, 0]], np.uint8)
    assert np.array_equal(DEF.brute_force(A, d), want)
    assert np.array_equal(DEF.meet_in_middle(A, d), want)


@pytest.mark.parametrize("seed", range(4))
def test_definition_methods_agree(seed):
    inst = I.small(77 + seed, 2, 20, 10)
    assert np.array_equal(DEF.brute_force(inst.A, inst.d), DEF.meet_in_middle(inst.A, inst.d))


def test_paper_example_is_feasible_by_construction():
    """Every generated instance contains its planted x (Sec. 1, QOBLIB)."""
    for inst in I.batch_m4_7(8):
        assert np.array_equal(inst.A.astype(np.int64) @ inst.planted, inst.d)


@pytest.mark.parametrize("inst", SMALL, ids=lambda x: f"{x.tag}_s{x.seed}")
def test_all_modes_equal_brute_force(inst):
    want = DEF.brute_force(inst.A, inst.d)
    assert any(np.array_equal(inst.planted, x) for x in want)
    _, kern, g = O.reduce(inst.A, inst.d)
    nodes = {}
    for hm, sym in MODES:
        r = O.enumerate(kern, g, inst.A, inst.d, hoelder=hm, sym=sym)
        assert np.array_equal(r.solutions, want), (hm, sym)
        nodes[(hm, sym)] = r.nodes
    for sym in (True, False):
        # the Hoelder cut prunes at least as much as the per-value filter,
        # which prunes at least as much as no Hoelder test at all
        assert nodes[(O.HOELDER_CUT, sym)] <= nodes[(O.HOELDER_FILTER, sym)] <= nodes[(O.HOELDER_OFF, sym)]
    # literal mode walks v and -v: at least as many nodes as sym mode
    for hm in (O.HOELDER_CUT, O.HOELDER_FILTER, O.HOELDER_OFF):
        assert nodes[(hm, False)] >= nodes[(hm, True)]


@pytest.mark.parametrize("inst", I.batch_m4_7(24)[:24:3], ids=lambda x: x.tag)
def test_batch_shapes_equal_meet_in_middle(inst):
    if inst.n > 40:
        pytest.skip("meet in the middle covers n <= 40")
    want = DEF.meet_in_middle(inst.A, inst.d)
    r = O.solve(inst.A, inst.d).result
    assert np.array_equal(r.solutions, want)


def _is_subset(a, b):
    sb = {bytes(x) for x in b}
    return all(bytes(x) in sb for x in a)


@pytest.mark.parametrize("inst", SMALL[:12], ids=lambda x: f"{x.tag}_s{x.seed}")
def test_summation_order_does_not_change_the_set(inst):
    """Reading R9: with the slack of R4 the l1 lane count only moves ties.
    Without the slack (paper-literal eps = 0) solutions, which lie exactly on
    both bounds (||v||^2 = n+1 = ||v||_1), can be rounded away: the result is
    then only a subset of the true set."""
    want = DEF.brute_force(inst.A, inst.d)
    _, kern, g = O.reduce(inst.A, inst.d)
    for lanes in (1, 2, 8, 16, 32):
        r = O.enumerate(kern, g, inst.A, inst.d, lanes=lanes, use_eps=True)
        assert np.array_equal(r.solutions, want), lanes
        r0 = O.enumerate(kern, g, inst.A, inst.d, lanes=lanes, use_eps=False)
        assert _is_subset(r0.solutions, want), lanes


def test_zero_slack_loses_solutions():
    """The reason for R4: on this instance eps = 0 drops true solutions."""
    inst = SMALL[0]
    want = DEF.brute_force(inst.A, inst.d)
    _, kern, g = O.reduce(inst.A, inst.d)
    r0 = O.enumerate(kern, g, inst.A, inst.d, lanes=1, use_eps=False)
    assert len(r0.solutions) < len(want)


@pytest.mark.parametrize("inst", [SMALL[1], SMALL[3], I.batch_m4_7(3)[2], I.batch_m4_7(7)[5]],
                         ids=lambda x: x.tag)
@pytest.mark.parametrize("k", [1, 3, 6])
def test_split_is_a_partition(inst, k):
    """Top-k split (the tree partition of Sec. 4): node totals and solutions
    of the top part plus all subtrees equal the unsplit run."""
    _, kern, g = O.reduce(inst.A, inst.d)
    dd = kern.shape[0]
    whole = O.enumerate(kern, g, inst.A, inst.d)
    split_level = dd - k
    top = O.enumerate(kern, g, inst.A, inst.d, split_level=split_level)
    total = top.nodes
    sols = [top.solutions]
    for p in top.prefixes:
        sub = O.enumerate(kern, g, inst.A, inst.d, sub_level=split_level - 1, prefix=p)
        total += sub.nodes
        sols.append(sub.solutions)
    assert total == whole.nodes
    allsol = O.sort_solutions(np.concatenate(sols))
    assert np.array_equal(allsol, whole.solutions)


def test_first_mode_returns_a_valid_solution():
    inst = I.batch_m4_7(3)[1]
    r = O.solve(inst.A, inst.d, first=True).result
    assert r.stopped and r.nsol == 1
    x = r.solutions[0].astype(np.int64)
    assert np.array_equal(inst.A.astype(np.int64) @ x, inst.d)


@pytest.mark.parametrize("k", [0, 1, 2], ids=lambda k: SMALL[k].tag)
def test_first_mode_stops_at_one_of_many(k):
    """First-solution mode (Sec. 1: any solution answers fMSP) on instances
    with 107-451 solutions: exactly one is reported, it is in the
    brute-force set, and the walk stops early."""
    inst = SMALL[k]
    want = DEF.brute_force(inst.A, inst.d)
    assert len(want) > 100
    full = O.solve(inst.A, inst.d).result
    r = O.solve(inst.A, inst.d, first=True).result
    assert r.stopped and r.nsol == 1
    assert any(np.array_equal(r.solutions[0], w) for w in want)
    assert r.nodes < full.nodes


def test_infeasible_instance_has_no_solution():
    """Cornuejols-Dawande right-hand side d_i = floor(sum_j a_ij / 2) with a
    parity twist that makes it infeasible: d odd where every a_ij is even."""
    rng = np.random.default_rng(5)
    A = 2 * rng.integers(0, 30, size=(2, 18)).astype(np.int32)
    d = (A.sum(axis=1) // 2) | 1
    assert len(DEF.brute_force(A, d)) == 0
    r = O.solve(A, d.astype(np.int64)).result
    assert r.nsol == 0 and r.nodes > 0
