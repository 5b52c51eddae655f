"""GPU parity of BKZ (Sec. 2's alternative to LLL for step 1) against the
oracle: the reduced kernel basis, its Gram-Schmidt tables and the BKZ
counters bit for bit, then the enumeration on it node for node."""
import numpy as np
import pytest

from oracle import definition as DEF
from oracle import oracle as O
from paper_2508_08702_gb300 import instances as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_08702_gb300 import build
    build.build()
    from oracle import build as ob
    ob.build()


SMALL = [I.small(1000 + s, m, n, D) for s in range(2)
         for (m, n, D) in [(2, 18, 12), (3, 20, 8), (4, 22, 6), (3, 21, 100), (1, 16, 60)]]
MIXED = SMALL + I.batch_m4_7(8)[:6]


def M():
    from paper_2508_08702_gb300 import msp
    return msp


@pytest.mark.parametrize("beta", [2, 4, 10, 20])
def test_bkz_basis_and_tables_bit_exact(beta):
    pk = I.pack(MIXED)
    ctx = M().Context(bkz_beta=beta, max_seconds=120.0)
    ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
    ctx.msp_reduce()
    res = ctx.msp_enumerate()
    for i, inst in enumerate(MIXED):
        _, kern, _ = O.reduce(inst.A, inst.d)
        ref = O.bkz(kern, beta)
        kb, mu, B, bhat = ctx.msp_export_gso(i)
        assert np.array_equal(kb, ref.kern), (i, beta)
        g = O.gso(ref.kern)
        assert np.array_equal(B, g.B) and np.array_equal(bhat, g.bhat), i
        assert np.array_equal(np.tril(mu), np.tril(g.mu)), i
        st = res.stats[i]
        assert (st["bkz_tours"], st["bkz_inserts"], st["bkz_nodes"]) == (ref.tours, ref.inserts, ref.nodes), i
    ctx.close()


def test_enumeration_on_bkz_basis_equals_oracle():
    res, sols, ctx = M().solve(MIXED, bkz_beta=10, lanes=8, max_seconds=120.0)
    for i, inst in enumerate(MIXED):
        _, kern, _ = O.reduce(inst.A, inst.d)
        kb = O.bkz(kern, 10).kern
        ref = O.enumerate(kb, O.gso(kb), inst.A, inst.d, lanes=8)
        assert res.stats[i]["nodes"] == ref.nodes, i
        assert np.array_equal(sols[i], ref.solutions), i
        if inst.n <= 24:
            assert np.array_equal(sols[i], DEF.brute_force(inst.A, inst.d)), i
    ctx.close()


def test_bkz_shrinks_the_tree_at_m7():
    insts = [x for x in I.batch_m4_7(16) if x.m == 7][:3]
    r0, _, c0 = M().solve(insts, max_seconds=120.0)
    r1, s1, c1 = M().solve(insts, bkz_beta=10, max_seconds=120.0)
    assert r1.total["nodes"] < 0.7 * r0.total["nodes"]
    for i, inst in enumerate(insts):
        assert any(np.array_equal(inst.planted, x) for x in s1[i])
    c0.close()
    c1.close()
