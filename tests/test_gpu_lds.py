"""GPU parity of the limited discrepancy search (Sec. 3) against the oracle.

One iteration with a fixed budget is deterministic: nodes, passed nodes,
leaves and the solutions with exactly that many discrepancies must equal the
oracle's, whatever the split and the walkers' interleaving.  The iterated
search must report every solution exactly once (all mode) and stop every
instance at the least budget that holds a solution (first mode)."""
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


def _oracle(inst, **kw):
    _, kern, g = O.reduce(inst.A, inst.d)
    return O.enumerate(kern, g, inst.A, inst.d, lanes=8, **kw)


@pytest.mark.parametrize("rank", [0, 1], ids=["flat", "rank"])
@pytest.mark.parametrize("k", [0, 1, 3, 6])
@pytest.mark.parametrize("depth", [0, 8, 24])
def test_one_iteration_equals_oracle(k, depth, rank):
    insts = MIXED if depth else SMALL   # one walker per instance without a split
    res, sols, ctx = M().solve(insts, order=M().MSP_LDS, lds_budget=k, split_depth=depth, lanes=8,
                               max_seconds=120.0, lds_rank=rank)
    for i, inst in enumerate(insts):
        ref = _oracle(inst, lds=k, lds_rank=bool(rank))
        st = res.stats[i]
        assert (st["nodes"], st["passed"], st["leaves"]) == (ref.nodes, ref.passed, ref.leaves), (i, k)
        assert np.array_equal(sols[i], ref.solutions), (i, k)
    ctx.close()


@pytest.mark.parametrize("rank", [0, 1], ids=["flat", "rank"])
def test_iterated_all_mode_reports_every_solution_once(rank):
    res, sols, ctx = M().solve(SMALL, order=M().MSP_LDS, lanes=8, max_seconds=120.0, lds_rank=rank)
    for i, inst in enumerate(SMALL):
        assert np.array_equal(sols[i], DEF.brute_force(inst.A, inst.d)), i
        _, kern, g = O.reduce(inst.A, inst.d)
        its = O.enumerate_lds(kern, g, inst.A, inst.d, lanes=8, lds_rank=bool(rank))
        assert res.stats[i]["lds_budget"] == len(its) - 1
        assert res.stats[i]["nodes"] == sum(r.nodes for r in its)
    ctx.close()


@pytest.mark.parametrize("rank", [0, 1], ids=["flat", "rank"])
def test_first_mode_stops_at_the_least_budget(rank):
    insts = [x for x in I.batch_m4_7(24) if x.m <= 6][:10]
    res, sols, ctx = M().solve(insts, mode=M().MSP_FIRST, order=M().MSP_LDS, lanes=8, max_seconds=120.0,
                               lds_rank=rank)
    for i, inst in enumerate(insts):
        _, kern, g = O.reduce(inst.A, inst.d)
        its = O.enumerate_lds(kern, g, inst.A, inst.d, lanes=8, first=True, lds_rank=bool(rank))
        assert res.stats[i]["lds_budget"] == len(its) - 1, i
        assert res.stats[i]["first_ms"] >= 0
        assert len(sols[i]) >= 1
        for x in sols[i].astype(np.int64):
            assert np.array_equal(inst.A.astype(np.int64) @ x, inst.d)
    ctx.close()


def test_lds_budget_cap_reports_ecap():
    """An iterated search that reaches opts.lds_max before the tree is
    exhausted says so (MSP_ECAP) instead of returning a partial set as
    complete."""
    inst = [x for x in I.batch_m4_7(24) if x.m == 5][0]
    _, kern, g = O.reduce(inst.A, inst.d)
    its = O.enumerate_lds(kern, g, inst.A, inst.d, lanes=8)
    assert len(its) >= 3   # the tree needs budget 2 or more
    res, sols, ctx = M().solve([inst], order=M().MSP_LDS, lanes=8, lds_max=1, max_seconds=120.0,
                               allow=(M().MSP_OK, M().MSP_ECAP))
    assert res.stats[0]["status"] == M().MSP_ECAP
    assert res.stats[0]["nodes"] == its[0].nodes + its[1].nodes
    ctx.close()


def test_lds_time_cap_and_order_errors():
    inst = [x for x in I.batch_m4_7(8) if x.m == 7][0]
    res, sols, ctx = M().solve([inst], order=M().MSP_LDS, time_cap_s=0.02, lanes=8,
                               allow=(M().MSP_OK, M().MSP_ETIMEOUT))
    for x in sols[0].astype(np.int64):
        assert np.array_equal(inst.A.astype(np.int64) @ x, inst.d)
    with pytest.raises(M().MspError):
        ctx.msp_run_async(M().MSP_FIRST, M().MSP_LDS)
    ctx.close()


@pytest.mark.parametrize("k", [1, 4])
def test_learned_order_inside_an_iteration_changes_no_node(k):
    """MSP_LDS_LEARNED takes an iteration's subtrees in the scorer's order:
    the same nodes, leaves and solutions as the oracle's iteration."""
    from oracle import mlp as R
    res, sols, ctx = M().solve(MIXED, order=M().MSP_LDS_LEARNED, scorer=R.init(9), lds_budget=k, lanes=8,
                               split_depth=8, max_seconds=120.0)
    for i, inst in enumerate(MIXED):
        ref = _oracle(inst, lds=k)
        st = res.stats[i]
        assert (st["nodes"], st["passed"], st["leaves"]) == (ref.nodes, ref.passed, ref.leaves), i
        assert np.array_equal(sols[i], ref.solutions), i
    ctx.close()


def test_learned_order_inside_the_search_finds_the_same_first_budget():
    from oracle import mlp as R
    insts = [x for x in I.batch_m4_7(24) if x.m <= 6][:8]
    res, sols, ctx = M().solve(insts, mode=M().MSP_FIRST, order=M().MSP_LDS_LEARNED, scorer=R.init(4), lanes=8,
                               max_seconds=120.0)
    for i, inst in enumerate(insts):
        _, kern, g = O.reduce(inst.A, inst.d)
        its = O.enumerate_lds(kern, g, inst.A, inst.d, lanes=8, first=True)
        assert res.stats[i]["lds_budget"] == len(its) - 1, i
        assert len(sols[i]) >= 1
        for x in sols[i].astype(np.int64):
            assert np.array_equal(inst.A.astype(np.int64) @ x, inst.d)
    ctx.close()
