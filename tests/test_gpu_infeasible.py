"""Cornuejols-Dawande instances on the GPU (Sec. 1: the original market split
problem, nothing planted, some instances infeasible): the all-solutions answer equals the
oracle's node for node -- for an infeasible instance that is the proof of
infeasibility -- and the first-solution modes (plain and LDS) end every
infeasible instance with no solution and no error."""
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


CD = I.cd_batch(3, 4) + I.cd_batch(4, 4) + I.cd_batch(5, 4) + I.cd_batch(6, 4)


def M():
    from paper_2508_08702_gb300 import msp
    return msp


def test_cd_all_solutions_equal_oracle():
    res, sols, ctx = M().solve(CD, lanes=8, max_seconds=120.0)
    infeasible = 0
    for i, inst in enumerate(CD):
        ref = O.solve(inst.A, inst.d, lanes=8).result
        assert res.stats[i]["status"] == 0
        assert res.stats[i]["nodes"] == ref.nodes, inst.tag
        assert np.array_equal(sols[i], ref.solutions), inst.tag
        if inst.n <= 40:
            assert np.array_equal(sols[i], DEF.meet_in_middle(inst.A, inst.d)), inst.tag
        infeasible += len(sols[i]) == 0
    assert infeasible >= 4
    ctx.close()


@pytest.mark.parametrize("order", ["plain", "lds"])
def test_cd_first_mode_ends_infeasible_instances(order):
    o = {"plain": M().MSP_PLAIN, "lds": M().MSP_LDS}[order]
    res, sols, ctx = M().solve(CD, mode=M().MSP_FIRST, order=o, lanes=8, max_seconds=120.0)
    for i, inst in enumerate(CD):
        feasible = O.solve(inst.A, inst.d, lanes=8).result.nsol > 0
        st = res.stats[i]
        assert st["status"] == 0, inst.tag
        if feasible:
            assert len(sols[i]) >= 1 and st["first_ms"] >= 0, inst.tag
            for x in sols[i].astype(np.int64):
                assert np.array_equal(inst.A.astype(np.int64) @ x, inst.d)
        else:
            assert len(sols[i]) == 0 and st["first_ms"] < 0, inst.tag
    ctx.close()
