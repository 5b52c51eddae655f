"""Pins for the oracle's lattice steps (Sec. 2, Eq. (2) and (4); Alg. 1 steps 1-3).

Everything here is checked against exact integer or rational arithmetic
done independently in the test, never against the oracle itself.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_08702_gb300 import instances as I


def exact_gso(vectors):
    """Gram-Schmidt of Eq. (4) in exact rationals: returns (mu, B)."""
    V = [[Fraction(int(x)) for x in v] for v in vectors]
    K = len(V)
    bh = []
    mu = [[Fraction(0)] * K for _ in range(K)]
    B = []
    for i in range(K):
        w = list(V[i])
        for j in range(i):
            if B[j] == 0:
                continue
            mu[i][j] = sum(a * b for a, b in zip(V[i], bh[j])) / B[j]
            w = [a - mu[i][j] * b for a, b in zip(w, bh[j])]
        bh.append(w)
        B.append(sum(a * a for a in w))
        mu[i][i] = Fraction(1)
    return mu, B, bh


def rank_exact(M):
    """Rank over Q by fraction Gaussian elimination."""
    R = [[Fraction(int(x)) for x in row] for row in M]
    rows, cols = len(R), len(R[0])
    r = 0
    for c in range(cols):
        p = next((i for i in range(r, rows) if R[i][c] != 0), None)
        if p is None:
            continue
        R[r], R[p] = R[p], R[r]
        for i in range(rows):
            if i != r and R[i][c] != 0:
                f = R[i][c] / R[r][c]
                R[i] = [a - f * b for a, b in zip(R[i], R[r])]
        r += 1
    return r


def det_bareiss(M):
    """Exact integer determinant (fraction-free Bareiss elimination)."""
    A = [[int(x) for x in row] for row in M]
    n = len(A)
    sign, prev = 1, 1
    for k in range(n - 1):
        if A[k][k] == 0:
            p = next((i for i in range(k + 1, n) if A[i][k] != 0), None)
            if p is None:
                return 0
            A[k], A[p] = A[p], A[k]
            sign = -sign
        for i in range(k + 1, n):
            for j in range(k + 1, n):
                A[i][j] = (A[i][j] * A[k][k] - A[i][k] * A[k][j]) // prev
        prev = A[k][k]
    return sign * A[n - 1][n - 1]


CASES = [I.single_m3()[0], I.small(11, 2, 14, 40), I.small(12, 4, 18, 30)]


@pytest.mark.parametrize("inst", CASES, ids=lambda x: x.tag)
def test_lattice_contains_planted_solution(inst):
    """Eq. (2): u = (1, x) gives (N(Ax - d); 2x - 1; 1) = (0; +-1; 1)."""
    b = O.build_lattice(inst.A, inst.d, N=1024)
    m, n = inst.m, inst.n
    assert b.shape == (n + 1, m + n + 1)
    u = np.concatenate([[1], inst.planted.astype(np.int64)])
    v = u @ b
    assert np.all(v[:m] == 0)
    assert np.array_equal(v[m:m + n], 2 * inst.planted.astype(np.int64) - 1)
    assert v[m + n] == 1
    # a non-solution combination leaves a nonzero N-scaled top part
    u2 = u.copy()
    u2[1] ^= 1
    assert np.any((u2 @ b)[:m] != 0)
    assert np.all(((u2 @ b)[:m]) % 1024 == 0)


@pytest.mark.parametrize("inst", CASES, ids=lambda x: x.tag)
def test_lll_is_unimodular_and_reduced(inst):
    b0 = O.build_lattice(inst.A, inst.d)
    red = O.lll(b0)
    b1 = red.basis
    m, n = inst.m, inst.n
    # rows m..m+n of the generator form an invertible square block S;
    # the transform U with b1 = U b0 is S1 S0^{-1}, which must be integral
    # with determinant +-1.
    S0 = b0[:, m:]
    S1 = b1[:, m:]
    sympy = pytest.importorskip("sympy")
    U = sympy.Matrix(S1.tolist()) * sympy.Matrix(S0.tolist()).inv()
    assert all(x.is_integer for x in U)
    assert abs(U.det()) == 1
    assert (sympy.Matrix(b1.tolist()) - U * sympy.Matrix(b0.tolist())).is_zero_matrix
    # LLL conditions in exact rationals (eta = 0.51, delta = 0.99, with a
    # relative slack of 1e-9 for the floating-point decisions)
    mu, B, _ = exact_gso(b1)
    K = len(B)
    for i in range(K):
        for j in range(i):
            assert abs(mu[i][j]) <= Fraction(51, 100) + Fraction(1, 10 ** 9)
    for k in range(1, K):
        lhs = B[k]
        rhs = (Fraction(99, 100) - mu[k][k - 1] ** 2) * B[k - 1]
        assert lhs >= rhs * (1 - Fraction(1, 10 ** 9))


@pytest.mark.parametrize("inst", CASES + I.batch_m4_7(6), ids=lambda x: x.tag)
def test_extraction_is_a_kernel_basis(inst):
    """Alg. 1 step 2: n - rank + 1 kept vectors, all in ker[A | -d]."""
    red = O.lll(O.build_lattice(inst.A, inst.d))
    kern = O.extract(red.basis, inst.m)
    Ad = np.concatenate([inst.A.astype(np.int64), -inst.d.reshape(-1, 1)], axis=1)
    rank = rank_exact(Ad.tolist())
    assert kern.shape == (inst.n + 1 - rank, inst.n + 1)
    # a kept vector (z; h) = (2u - u0 1; u0) with A u = d u0, i.e.
    # A z = (2 d - A 1) h
    A = inst.A.astype(np.int64)
    for v in kern.astype(np.int64):
        z, h = v[:-1], v[-1]
        assert np.array_equal(A @ z, (2 * inst.d - A.sum(axis=1)) * h)
        assert np.all((z + h) % 2 == 0)
    # the kept vectors are linearly independent
    assert rank_exact(kern.tolist()) == kern.shape[0]


@pytest.mark.parametrize("inst", CASES, ids=lambda x: x.tag)
def test_gso_against_exact_rationals(inst):
    """Eq. (4): FP64 tables agree with exact Gram-Schmidt; prod B = det(Gram)."""
    _, kern, g = O.reduce(inst.A, inst.d)
    mu, B, bh = exact_gso(kern)
    dd, dim = kern.shape
    for i in range(dd):
        assert g.B[i] == pytest.approx(float(B[i]), rel=1e-11)
        for j in range(i):
            assert g.mu[i, j] == pytest.approx(float(mu[i][j]), rel=1e-9, abs=1e-12)
        for c in range(dim):
            assert g.bhat[i, c] == pytest.approx(float(bh[i][c]), rel=1e-9, abs=1e-11)
    G = (kern.astype(np.int64) @ kern.astype(np.int64).T).tolist()
    det = det_bareiss(G)
    assert det > 0
    logprod = float(np.sum(np.log(g.B)))
    assert logprod == pytest.approx(float(np.log(float(det))), rel=1e-12, abs=1e-9)
    # reconstruction b_i = bhat_i + sum_{j<i} mu_ij bhat_j, and orthogonality
    rec = np.tril(g.mu, -1) @ g.bhat + g.bhat
    assert np.max(np.abs(rec - kern)) < 1e-9
    Gh = g.bhat @ g.bhat.T
    off = Gh - np.diag(np.diag(Gh))
    assert np.max(np.abs(off)) < 1e-9 * np.max(g.B)


def test_lll_terminates_on_large_shapes():
    for inst in I.m12_n110(1) + I.m9_n80(1):
        red = O.lll(O.build_lattice(inst.A, inst.d))
        kern = O.extract(red.basis, inst.m)
        assert kern.shape == (inst.n - inst.m + 1, inst.n + 1)
