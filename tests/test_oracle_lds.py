"""Pins for the oracle's limited discrepancy search (Sec. 3, Harvey and
Ginsberg's scheme over Algorithm 1's value order).

Iteration k visits the paths with at most k discrepancies and reports the
leaves with exactly k.  Two readings of a discrepancy's cost: flat (every
value after the first of a level's walk costs one) and rank (the value at
position p of the walk costs p).  Pinned against things the oracle's C code
does not compute itself:
  * the discrepancy of every solution, derived here from its lattice
    coordinates (least squares on the kernel basis) and the exact rational
    Gram-Schmidt centres, matches the iteration that reports it (a centre
    that is exactly a half-integer may round either way in FP64, so such a
    level counts as either; under the rank reading a value v reached after
    a one-direction switch sits between |v - u^1| and its zig-zag index - 1);
  * the iterations partition the brute-force solution set;
  * with a budget no path can exhaust, iteration k is plain depth-first
    search node for node;
  * node counts grow with k; a split run plus its subtrees equals the whole
    iteration (so a prefix's discrepancy is rebuilt correctly).
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import definition as DEF
from oracle import oracle as O
from paper_2508_08702_gb300 import instances as I

CASES = [I.small(1000 + s, m, n, D) for s in range(3)
         for (m, n, D) in [(2, 18, 12), (3, 20, 8), (4, 22, 6), (3, 21, 100)]]


def exact_mu(kern):
    """Gram-Schmidt coefficients in exact rationals from the integer Gram matrix."""
    b = [[int(v) for v in row] for row in kern]
    dd = len(b)
    G = [[sum(x * y for x, y in zip(b[i], b[j])) for j in range(dd)] for i in range(dd)]
    mu = [[Fraction(0)] * dd for _ in range(dd)]
    B = [Fraction(0)] * dd
    for i in range(dd):
        for j in range(i):
            mu[i][j] = (G[i][j] - sum(mu[j][k] * mu[i][k] * B[k] for k in range(j))) / B[j]
        B[i] = Fraction(G[i][i]) - sum(mu[i][k] ** 2 * B[k] for k in range(i))
    return mu


def zigzag_index(v, u1, s):
    """Index (1-based) of v in the zig-zag u1, u1+s, u1-s, u1+2s, ..."""
    if v == u1:
        return 1
    return 2 * abs(v - u1) + (0 if (v - u1) * s > 0 else 1)


def rank_range(v, c, firsts):
    """(least, most) position of v in the walk of a level with centre c."""
    lo = hi = None
    for u1 in firsts:
        s = 1 if c >= u1 else -1
        a, b = abs(v - u1), zigzag_index(v, u1, s) - 1
        lo = a if lo is None else min(lo, a)
        hi = b if hi is None else max(hi, b)
    return lo, hi


def discrepancy_of(x, kern, mu, sym=True, rank=False):
    """(least, most) discrepancies of the path of solution x.  Flat: levels
    where u_t is not the rounded centre (0 on the all-zero top levels in sym
    mode).  Rank: the sum of the positions of u_t in their levels' walks.  A
    centre that is a half-integer accepts both neighbours."""
    v = np.concatenate([2 * x.astype(np.int64) - 1, [1]])
    u, *_ = np.linalg.lstsq(kern.T.astype(float), v.astype(float), rcond=None)
    u = np.rint(u).astype(np.int64)
    assert np.array_equal(u @ kern.astype(np.int64), v)
    nz = np.nonzero(u)[0]
    if sym and u[nz[-1]] < 0:
        u = -u
    dd = len(u)
    lo = hi = 0
    zero = True
    for t in range(dd - 1, -1, -1):
        if zero and sym:
            firsts = {0}
            c = None
        else:
            c = -sum(int(u[i]) * mu[i][t] for i in range(t + 1, dd))
            fl = c.numerator // c.denominator
            firsts = {fl, fl + 1} if c - fl == Fraction(1, 2) else {round(c)}
        if rank:
            if c is None:   # 0, 1, 2, ... from the start
                a = b = int(u[t])
            else:
                a, b = rank_range(int(u[t]), c, firsts)
            lo += a
            hi += b
        else:
            off = int(u[t]) not in firsts
            lo += off
            hi += off or len(firsts) > 1
        zero = zero and u[t] == 0
    return lo, hi


@pytest.mark.parametrize("rank", [False, True], ids=["flat", "rank"])
@pytest.mark.parametrize("inst", CASES, ids=lambda x: x.tag)
def test_iterations_partition_the_solution_set(inst, rank):
    _, kern, g = O.reduce(inst.A, inst.d)
    its = O.enumerate_lds(kern, g, inst.A, inst.d, lds_rank=rank)
    assert its[-1].lds_cuts == 0
    want = DEF.brute_force(inst.A, inst.d)
    got = [s for r in its for s in r.solutions]
    assert len(got) == len(want)
    assert np.array_equal(O.sort_solutions(np.array(got, np.uint8).reshape(-1, inst.n)), want)
    mu = exact_mu(kern)
    for k, r in enumerate(its):
        for x in r.solutions:
            lo, hi = discrepancy_of(x, kern, mu, rank=rank)
            assert lo <= k <= hi
    nodes = [r.nodes for r in its]
    assert nodes == sorted(nodes)


@pytest.mark.parametrize("rank", [False, True], ids=["flat", "rank"])
@pytest.mark.parametrize("inst", CASES[:6] + [I.batch_m4_7(3)[2]], ids=lambda x: x.tag)
def test_unbounded_budget_is_depth_first_search(inst, rank):
    _, kern, g = O.reduce(inst.A, inst.d)
    dfs = O.enumerate(kern, g, inst.A, inst.d)
    big = O.enumerate(kern, g, inst.A, inst.d, lds=1 << 20, lds_rank=rank)
    assert big.lds_cuts == 0
    assert (big.nodes, big.passed, big.leaves) == (dfs.nodes, dfs.passed, dfs.leaves)
    assert big.nsol == 0   # no path carries 2^20 discrepancies


@pytest.mark.parametrize("rank", [False, True], ids=["flat", "rank"])
def test_first_solution_comes_at_the_least_discrepancy(rank):
    inst = I.batch_m4_7(64)[18]   # m = 5, D = 50: several solutions
    _, kern, g = O.reduce(inst.A, inst.d)
    sols = DEF.meet_in_middle(inst.A, inst.d)
    mu = exact_mu(kern)
    ranges = [discrepancy_of(x, kern, mu, rank=rank) for x in sols]
    its = O.enumerate_lds(kern, g, inst.A, inst.d, first=True, lds_rank=rank)
    assert min(lo for lo, _ in ranges) <= len(its) - 1 <= min(hi for _, hi in ranges)
    assert its[-1].nsol == 1 and all(r.nsol == 0 for r in its[:-1])


@pytest.mark.parametrize("rank", [False, True], ids=["flat", "rank"])
@pytest.mark.parametrize("inst", [CASES[1], CASES[2], I.batch_m4_7(3)[2]], ids=lambda x: x.tag)
@pytest.mark.parametrize("k,depth", [(1, 3), (2, 5), (4, 6)])
def test_split_iteration_is_a_partition(inst, k, depth, rank):
    _, kern, g = O.reduce(inst.A, inst.d)
    dd = kern.shape[0]
    whole = O.enumerate(kern, g, inst.A, inst.d, lds=k, lds_rank=rank)
    sl = dd - depth
    top = O.enumerate(kern, g, inst.A, inst.d, lds=k, split_level=sl, lds_rank=rank)
    total, sols = top.nodes, [top.solutions]
    for p in top.prefixes:
        sub = O.enumerate(kern, g, inst.A, inst.d, lds=k, sub_level=sl - 1, prefix=p, lds_rank=rank)
        total += sub.nodes
        sols.append(sub.solutions)
    assert total == whole.nodes
    assert np.array_equal(O.sort_solutions(np.concatenate(sols)), whole.solutions)


@pytest.mark.parametrize("inst", CASES[:8] + [I.batch_m4_7(64)[18]], ids=lambda x: x.tag)
def test_rank_paths_are_a_subset_of_flat_paths(inst):
    """A value other than the first costs at least one under the rank
    reading, so with the same budget every path the rank iteration walks the
    flat one walks too: fewer nodes, and the solutions reported up to budget
    k are a subset of the flat ones (equal once both trees are exhausted)."""
    _, kern, g = O.reduce(inst.A, inst.d)
    got_r, got_f = set(), set()
    for k in range(5):
        r = O.enumerate(kern, g, inst.A, inst.d, lds=k, lds_rank=True)
        f = O.enumerate(kern, g, inst.A, inst.d, lds=k, lds_rank=False)
        assert r.nodes <= f.nodes and r.passed <= f.passed, k
        got_r |= {x.tobytes() for x in r.solutions}
        got_f |= {x.tobytes() for x in f.solutions}
        assert got_r <= got_f, k
    all_r = {x.tobytes() for it in O.enumerate_lds(kern, g, inst.A, inst.d, lds_rank=True) for x in it.solutions}
    all_f = {x.tobytes() for it in O.enumerate_lds(kern, g, inst.A, inst.d, lds_rank=False) for x in it.solutions}
    assert all_r == all_f
