"""GPU tests of the replica portfolio (Sec. 4: several randomly shuffled
input orders searched at once).  Each replica's tree is the oracle's tree
of the shuffled instance, so a group's node count is the sum of the
oracle's over the replicas, and its solutions -- put back in the caller's
order -- are the instance's solution set."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import replicas as RP
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


def M():
    from paper_2508_08702_gb300 import msp
    return msp


INSTS = [I.small(1000 + s, m, n, D) for s in range(2) for (m, n, D) in [(2, 18, 12), (3, 20, 8), (4, 22, 6)]] + \
        [I.bounded(700, 2, 14, 40, (1, 2, 3)), I.bounded(701, 3, 18, 30, (1, 2, 3))]


def _replica(inst, g, k):
    p = RP.permutation(inst.n, g, k)
    r = None if inst.r is None else inst.r[p]
    return inst.A[:, p], r


@pytest.mark.parametrize("R", [1, 3])
def test_all_mode_groups_equal_oracle(R):
    res, sols, ctx = M().solve(INSTS, lanes=8, replicas=R, max_seconds=120.0)
    assert len(res.stats) == len(INSTS)
    for g, inst in enumerate(INSTS):
        want = O.solve(inst.A, inst.d, r=inst.r, lanes=8).result.solutions
        nodes = 0
        for k in range(R):
            A, r = _replica(inst, g, k)
            nodes += O.solve(A, inst.d, r=r, lanes=8).result.nodes
        assert res.stats[g]["nodes"] == nodes, g
        assert np.array_equal(sols[g], want), g
        assert res.stats[g]["solutions"] == len(want)
    ctx.close()


def test_first_mode_with_replicas():
    insts = [x for x in I.batch_m4_7(64) if x.m == 7][:6]
    res, sols, ctx = M().solve(insts, mode=M().MSP_FIRST, replicas=4, max_seconds=120.0)
    for g, inst in enumerate(insts):
        assert res.stats[g]["status"] == 0
        assert res.stats[g]["first_ms"] >= 0 and len(sols[g]) >= 1
        for x in sols[g].astype(np.int64):
            assert np.array_equal(inst.A.astype(np.int64) @ x, inst.d)
    ctx.close()


def test_lds_with_replicas_stops_at_the_least_budget_of_the_group():
    insts = [x for x in I.batch_m4_7(24) if x.m <= 6][:5]
    R = 3
    res, sols, ctx = M().solve(insts, mode=M().MSP_FIRST, order=M().MSP_LDS, lanes=8, replicas=R,
                               max_seconds=120.0)
    for g, inst in enumerate(insts):
        budgets = []
        for k in range(R):
            A, _ = _replica(inst, g, k)
            _, kern, gs = O.reduce(A, inst.d)
            budgets.append(len(O.enumerate_lds(kern, gs, A, inst.d, lanes=8, first=True)) - 1)
        assert res.stats[g]["lds_budget"] == min(budgets), (g, budgets)
        assert len(sols[g]) >= 1
    ctx.close()
