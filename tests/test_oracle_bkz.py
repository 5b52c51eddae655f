"""Pins for the oracle's BKZ reduction of the kernel basis (Sec. 2 allows
block reduction in place of LLL for step 1).

Checked against things the C code does not compute itself:
  * the reduced basis spans the same lattice: an integer matrix U with
    |det U| = 1 maps the LLL basis onto it (exact integer arithmetic here);
  * Gram-Schmidt volume is preserved (product of B_i = det of the Gram
    matrix, by exact Bareiss elimination);
  * BKZ-reducedness: in every block the first projected vector is within
    delta of the block's shortest nonzero projected vector, found here by an
    independent exact-rational search on small lattices;
  * with beta = dd the first vector is a shortest vector of the lattice;
  * on instances whose LLL basis is not block-reduced and does not start
    with a shortest vector, BKZ inserts vectors and repairs both;
  * enumeration on the BKZ basis finds the brute-force solution set.
"""
from fractions import Fraction
import itertools

import numpy as np
import pytest

from oracle import definition as DEF
from oracle import oracle as O
from paper_2508_08702_gb300 import instances as I

CASES = [I.small(1000 + s, m, n, D) for s in range(3)
         for (m, n, D) in [(2, 18, 12), (3, 20, 8), (4, 22, 6), (3, 21, 100)]]


def bareiss_det(M):
    A = [[int(x) for x in row] for row in M]
    n = len(A)
    sign, prev = 1, 1
    for k in range(n - 1):
        if A[k][k] == 0:
            for i in range(k + 1, n):
                if A[i][k] != 0:
                    A[k], A[i] = A[i], A[k]
                    sign = -sign
                    break
            else:
                return 0
        for i in range(k + 1, n):
            for j in range(k + 1, n):
                A[i][j] = (A[i][j] * A[k][k] - A[i][k] * A[k][j]) // prev
        prev = A[k][k]
    return sign * A[-1][-1]


def exact_gso(b):
    b = [[int(v) for v in row] for row in b]
    dd = len(b)
    G = [[sum(x * y for x, y in zip(b[i], b[j])) for j in range(dd)] for i in range(dd)]
    mu = [[Fraction(0)] * dd for _ in range(dd)]
    B = [Fraction(0)] * dd
    for i in range(dd):
        for j in range(i):
            mu[i][j] = (G[i][j] - sum(mu[j][q] * mu[i][q] * B[q] for q in range(j))) / B[j]
        B[i] = Fraction(G[i][i]) - sum(mu[i][q] ** 2 * B[q] for q in range(i))
    return mu, B


def block_shortest(mu, B, k, h):
    """Squared length of the shortest nonzero vector of the projected block
    [k, h), by exact Fincke-Pohst search (rational arithmetic)."""
    best = B[k]
    n = h - k
    u = [0] * n

    def rec(t, rho):
        nonlocal best
        c = -sum(u[i] * mu[k + i][k + t] for i in range(t + 1, n))
        # all integers x with rho + (x - c)^2 B <= best
        import math
        span = (best - rho) / B[k + t]
        if span < 0:
            return
        r = Fraction(math.isqrt(int(span.numerator // span.denominator) + 1) + 1)
        lo, hi = int(c - r) - 1, int(c + r) + 1
        for x in range(lo, hi + 1):
            d = rho + (x - c) ** 2 * B[k + t]
            if d > best:
                continue
            u[t] = x
            if t == 0:
                if any(u) and d < best:
                    best = d
            else:
                rec(t - 1, d)
            u[t] = 0

    rec(n - 1, Fraction(0))
    return best


# Instances on which LLL leaves work for the block search: some block of
# width 4 of the LLL basis is not delta-reduced, and its first vector is not
# a shortest one (squared norms 24 against 20, and 73 against 25).  On the
# small-D cases the LLL basis often passes these checks already and BKZ
# inserts nothing, so only these show that the block search finds what is
# missing and that its insertions keep the lattice.
HARD = [I.small(2003, 2, 20, 200), I.small(2005, 3, 24, 1000)]


def assert_same_lattice(kern, kb):
    """kb = U kern with U integral and |det U| = 1, and equal Gram volumes."""
    kb = kb.astype(np.int64)
    U = np.rint(kb.astype(float) @ np.linalg.pinv(kern.astype(float))).astype(np.int64)
    assert np.array_equal(U @ kern.astype(np.int64), kb)
    assert abs(bareiss_det(U)) == 1
    G0 = kern.astype(object) @ kern.astype(object).T
    G1 = kb.astype(object) @ kb.astype(object).T
    assert bareiss_det(G0) == bareiss_det(G1)


@pytest.mark.parametrize("inst", CASES + HARD, ids=lambda x: x.tag)
@pytest.mark.parametrize("beta", [4, 10])
def test_same_lattice_and_volume(inst, beta):
    _, kern, _ = O.reduce(inst.A, inst.d)
    r = O.bkz(kern, beta)
    if any(inst is h for h in HARD):
        assert r.inserts > 0
    assert_same_lattice(kern, r.kern)


@pytest.mark.parametrize("inst", CASES[:4], ids=lambda x: x.tag)
def test_blocks_are_reduced(inst):
    beta, delta = 4, 0.99
    _, kern, _ = O.reduce(inst.A, inst.d)
    kb = O.bkz(kern, beta, delta=delta).kern
    mu, B = exact_gso(kb)
    dd = len(B)
    for k in range(dd - 1):
        h = min(k + beta, dd)
        lam = block_shortest(mu, B, k, h)
        assert delta * float(B[k]) <= float(lam) * (1 + 1e-12), k


def test_full_block_gives_a_shortest_vector():
    inst = I.small(1001, 2, 12, 6)
    _, kern, _ = O.reduce(inst.A, inst.d)
    dd = kern.shape[0]
    kb = O.bkz(kern, dd, delta=0.999999).kern
    mu, B = exact_gso(kb)
    lam = block_shortest(mu, B, 0, dd)
    assert float(B[0]) <= float(lam) / 0.999999 * (1 + 1e-12)


@pytest.mark.parametrize("inst", HARD, ids=lambda x: x.tag)
def test_block_search_repairs_what_lll_leaves(inst):
    beta, delta = 4, Fraction(99, 100)
    _, kern, _ = O.reduce(inst.A, inst.d)
    mu0, B0 = exact_gso(kern)
    dd = len(B0)
    assert any(delta * B0[k] > block_shortest(mu0, B0, k, min(k + beta, dd)) for k in range(dd - 1))
    r = O.bkz(kern, beta, delta=0.99)
    assert r.inserts > 0
    mu, B = exact_gso(r.kern)
    for k in range(dd - 1):
        lam = block_shortest(mu, B, k, min(k + beta, dd))
        assert float(delta * B[k]) <= float(lam) * (1 + 1e-12), k


@pytest.mark.parametrize("inst", HARD, ids=lambda x: x.tag)
def test_full_block_finds_the_shortest_vector_lll_missed(inst):
    _, kern, _ = O.reduce(inst.A, inst.d)
    mu0, B0 = exact_gso(kern)
    dd = len(B0)
    lam = block_shortest(mu0, B0, 0, dd)
    assert B0[0] > lam
    kb = O.bkz(kern, dd, delta=0.999999).kern
    # ||b_0||^2 is an integer and at most lam / 0.999999, so it equals lam
    assert int(np.dot(kb[0].astype(np.int64), kb[0].astype(np.int64))) == lam
    assert_same_lattice(kern, kb)


@pytest.mark.parametrize("inst", CASES, ids=lambda x: x.tag)
def test_enumeration_on_bkz_basis_finds_every_solution(inst):
    _, kern, _ = O.reduce(inst.A, inst.d)
    kb = O.bkz(kern, 10).kern
    g = O.gso(kb)
    r = O.enumerate(kb, g, inst.A, inst.d)
    assert np.array_equal(r.solutions, DEF.brute_force(inst.A, inst.d))
