"""The oracle's node counts pinned to exact counts taken from the definitions
of Algorithm 1's pruning conditions.

With the Hoelder cut off (HOELDER_OFF), or applied as a filter only
(HOELDER_FILTER: a node that fails Theorem 2's bound is not expanded and its
level goes on), the nodes Algorithm 1 evaluates do not depend on the order
of the walk.  Below every expanded prefix (u_{t+1}, ..., u_{d-1}) the
passing values of level t are the integers u with

    rho_t = (u - c_t)^2 B_t + rho_{t+1} <= R + eps,   c_t = -sum_{i>t} u_i mu_it

(an interval around the centre c_t, Sec. 2), and the walk evaluates one
value more: it visits values by nondecreasing distance from c_t, so the
first failure is the first value outside the interval.  A passing node at
t > 0 is expanded (all of it with HOELDER_OFF; with HOELDER_FILTER only if
rho_t <= ||w^(t)||_1 + eps, w^(t) = sum_{i>=t} (u_i - c_i) bhat_i, Theorem 2).
Symmetry (R6) restricts a level under an all-zero prefix to u >= 0.

Everything here is an exact rational (fractions.Fraction) from an exact
Gram-Schmidt of the kernel basis, computed without the oracle's tables or
its FP64 arithmetic, so a dropped term, a wrong sign or index in the
oracle's centre, partial norm, w update or l1 norm changes the counts.
Instances are kept away from the bounds: no exact rho_t or l1 bound lies
within a relative 1e-9 of its threshold (the oracle's FP64 rounding is far
smaller), which the test checks."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_08702_gb300 import instances as I

GUARD = Fraction(1, 10**9)


def exact_gso(kern):
    d, dim = kern.shape
    b = [[Fraction(int(v)) for v in row] for row in kern]
    bh, B = [], []
    mu = [[Fraction(0)] * d for _ in range(d)]
    for i in range(d):
        v = list(b[i])
        for j in range(i):
            mu[i][j] = sum(b[i][c] * bh[j][c] for c in range(dim)) / B[j]
            v = [v[c] - mu[i][j] * bh[j][c] for c in range(dim)]
        bh.append(v)
        B.append(sum(x * x for x in v))
    return mu, B, bh


class _Over(Exception):
    pass


def exact_counts(kern, filt, sym, mistake=None, limit=None):
    """Exact (nodes, passed, leaves) and the smallest relative distance of an
    exact value to its threshold; with `limit`, stops (nodes = limit + 1)
    once more nodes than that are counted."""
    d, dim = kern.shape
    mu, B, bh = exact_gso(kern)
    R = Fraction(dim)                       # (n + 1) r_max^2, r_max = 1
    eps = R / 2**20                         # R4
    Rb = R + eps
    cnt = {"nodes": 0, "passed": 0, "leaves": 0}
    closest = [Fraction(1)]                 # smallest relative distance to a threshold
    u = [0] * d

    def near(a, thr):
        if thr != 0:
            closest[0] = min(closest[0], abs(a - thr) / abs(thr))

    def level(t, rho_p, wp, zero):
        c = -sum(u[i] * mu[i][t] for i in range(t + 1, d))
        if mistake == "sign":
            c = -c
        elif mistake == "index":
            c = -sum(u[i] * mu[t + 1][t] for i in range(t + 1, d)) if t + 1 < d else c
        def rho_of(v):
            return (v - c) ** 2 * B[t] + (0 if mistake == "drop" else rho_p)
        vals = []
        if zero and sym:                    # R6: u = 0, 1, 2, ... only
            v = 0
            while rho_of(v) <= Rb:
                vals.append(v)
                v += 1
            near(rho_of(v), Rb)
        else:
            lo = math.floor(c)
            v = lo
            while rho_of(v) <= Rb:
                vals.append(v)
                v -= 1
            near(rho_of(v), Rb)
            v = lo + 1
            while rho_of(v) <= Rb:
                vals.append(v)
                v += 1
            near(rho_of(v), Rb)
        cnt["nodes"] += len(vals) + 1
        cnt["passed"] += len(vals)
        if limit is not None and cnt["nodes"] > limit:
            raise _Over()
        for v in vals:
            rho = rho_of(v)
            near(rho, Rb)
            if t == 0:
                cnt["leaves"] += 1
                continue
            u[t] = v
            x = v - c
            w = [wp[k] + x * bh[t][k] for k in range(dim)]
            if filt:
                h = sum(abs(z) for z in w) + eps
                near(rho, h)
                if rho > h:
                    continue
            level(t - 1, rho, w, zero and v == 0)
        u[t] = 0

    try:
        level(d - 1, Fraction(0), [Fraction(0)] * dim, True)
    except _Over:
        cnt["nodes"] = limit + 1
    return cnt, closest[0]


CASES = [I.small(1400 + s, m, n, D) for s, (m, n, D) in
         enumerate([(2, 16, 12), (3, 18, 8), (2, 18, 30), (4, 20, 6), (3, 20, 100), (1, 14, 60), (2, 22, 20),
                    (3, 24, 10)])]


@pytest.mark.parametrize("inst", CASES, ids=lambda x: x.tag)
@pytest.mark.parametrize("sym", [False, True], ids=["literal", "sym"])
@pytest.mark.parametrize("mode", [O.HOELDER_OFF, O.HOELDER_FILTER], ids=["off", "filter"])
def test_counts_equal_the_definition(inst, sym, mode):
    _, kern, g = O.reduce(inst.A, inst.d)
    ref, gap = exact_counts(kern, mode == O.HOELDER_FILTER, sym)
    assert gap > GUARD, gap
    for lanes in (1, 8):
        r = O.enumerate(kern, g, inst.A, inst.d, hoelder=mode, sym=sym, lanes=lanes)
        assert (r.nodes, r.passed, r.leaves) == (ref["nodes"], ref["passed"], ref["leaves"]), lanes


@pytest.mark.parametrize("mistake", ["sign", "index", "drop"])
def test_a_misread_centre_or_norm_changes_the_counts(mistake):
    """The counts tell these readings apart: a centre of the wrong sign, a
    centre from the wrong mu entry, a partial norm without rho_{t+1}."""
    inst = CASES[1]
    _, kern, g = O.reduce(inst.A, inst.d)
    r = O.enumerate(kern, g, inst.A, inst.d, hoelder=O.HOELDER_OFF, sym=False, lanes=8)
    bad, _ = exact_counts(kern, False, False, mistake, limit=10 * r.nodes)
    assert (r.nodes, r.passed, r.leaves) != (bad["nodes"], bad["passed"], bad["leaves"])


def test_filter_prunes_and_the_cut_prunes_more():
    """Theorem 2's bound removes nodes (the filter below the plain norm
    test, the one-direction cut below the filter) and no solution."""
    inst = CASES[3]
    _, kern, g = O.reduce(inst.A, inst.d)
    off, _ = exact_counts(kern, False, True)
    filt, _ = exact_counts(kern, True, True)
    assert filt["nodes"] < off["nodes"]
    cut = O.enumerate(kern, g, inst.A, inst.d, hoelder=O.HOELDER_CUT)
    assert cut.nodes <= filt["nodes"]
    assert np.array_equal(cut.solutions, O.enumerate(kern, g, inst.A, inst.d, hoelder=O.HOELDER_OFF).solutions)


def exact_prefixes(kern, split_level, sym):
    """Every prefix (u_split_level, ..., u_{d-1}) whose partial norms stay
    within R + eps at each of its levels, with rho at the split level, in
    exact rationals (the split of the tree at `split_level` with the Hoelder
    test off)."""
    mu, B, _ = exact_gso(kern)
    dd = len(B)
    Rb = Fraction(kern.shape[1]) * (1 + Fraction(1, 2 ** 20))
    u = [0] * dd
    out = {}

    def rec(t, rho, zero):
        c = -sum(u[i] * mu[i][t] for i in range(t + 1, dd))
        span = (Rb - rho) / B[t]
        if span < 0:
            return
        r = math.isqrt(span.numerator // span.denominator) + 1
        lo, hi = math.floor(c) - r - 1, math.ceil(c) + r + 1
        if zero and sym:
            lo = max(lo, 0)
        for x in range(lo, hi + 1):
            d = rho + (x - c) ** 2 * B[t]
            if d > Rb:
                continue
            u[t] = x
            if t == split_level:
                out[tuple(u[split_level:])] = d
            else:
                rec(t - 1, d, zero and x == 0)
        u[t] = 0

    rec(dd - 1, Fraction(0), True)
    return out


@pytest.mark.parametrize("inst", CASES[:4], ids=lambda x: x.tag)
@pytest.mark.parametrize("sym", [False, True], ids=["literal", "sym"])
def test_split_prefixes_and_their_norms_are_exact(inst, sym):
    """The split the GPU splitter is compared with: with the Hoelder test
    off the recorded prefixes are exactly the paths inside the norm bound,
    and each recorded rho is the exact partial norm of its prefix; with the
    default one-direction cut every recorded prefix is one of those paths,
    with the same exact rho."""
    _, kern, g = O.reduce(inst.A, inst.d)
    dd = kern.shape[0]
    for split_level in (dd - 3, dd - 6):
        want = exact_prefixes(kern, split_level, sym)
        for hoelder in (O.HOELDER_OFF, O.HOELDER_CUT):
            top = O.enumerate(kern, g, inst.A, inst.d, hoelder=hoelder, sym=sym, split_level=split_level)
            got = {tuple(int(v) for v in p[split_level:]): float(r) for p, r in zip(top.prefixes, top.prefix_rho)}
            assert len(got) == top.nprefix
            if hoelder == O.HOELDER_OFF:
                assert set(got) == set(want)
            else:
                assert set(got) <= set(want)
            for key, rho in got.items():
                assert rho == pytest.approx(float(want[key]), rel=1e-12, abs=1e-12), key
