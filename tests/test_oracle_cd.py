"""Cornuejols-Dawande instances (Sec. 1: d_i = floor(sum_j a_ij / 2), nothing
planted, some of them infeasible): the oracle's answer -- the complete solution set, usually
empty -- equals brute force / meet-in-the-middle, and the limited
discrepancy search proves infeasibility by exhausting the tree."""
import numpy as np
import pytest

from oracle import definition as DEF
from oracle import oracle as O
from paper_2508_08702_gb300 import instances as I

CD = I.cd_batch(3, 4) + I.cd_batch(4, 4) + I.cd_batch(5, 4)


@pytest.mark.parametrize("inst", CD, ids=lambda x: x.tag)
def test_cd_solution_sets(inst):
    want = DEF.brute_force(inst.A, inst.d) if inst.n <= 24 else DEF.meet_in_middle(inst.A, inst.d)
    assert np.array_equal(O.solve(inst.A, inst.d).result.solutions, want)


def test_cd_batch_has_infeasible_instances():
    assert sum(O.solve(x.A, x.d).result.nsol == 0 for x in CD) >= 4


@pytest.mark.parametrize("inst", [x for x in CD if x.m == 5], ids=lambda x: x.tag)
def test_lds_first_mode_on_cd(inst):
    _, kern, g = O.reduce(inst.A, inst.d)
    its = O.enumerate_lds(kern, g, inst.A, inst.d, first=True)
    dfs = O.enumerate(kern, g, inst.A, inst.d)
    if dfs.nsol == 0:   # infeasible: the last iteration held nothing back and found nothing
        assert its[-1].lds_cuts == 0 and all(r.nsol == 0 for r in its)
    else:
        assert its[-1].nsol == 1
