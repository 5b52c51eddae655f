"""Pins of the stored m = 9, n = 80, D = 100 results (tests/golden/), which
the GPU's complete runs are compared with: every stored x solves A x = d
exactly (the fMSP definition of Sec. 1) for the instance regenerated from its
seed, the planted x is among them, the sets are sorted and free of
duplicates, and every instance of the workload is present."""
import numpy as np

from paper_2508_08702_gb300 import instances as I
from tests.golden import m9_golden


def test_stored_solutions_solve_the_instances():
    g = m9_golden.load()
    insts = I.m9_n80(8)
    assert g.lanes == 16 and sorted(g.instances) == [x.seed for x in insts]
    for inst in insts:
        st = g.instances[inst.seed]
        X = st.solutions.astype(np.int64)
        assert X.shape[1] == inst.n and len(X) >= 1
        assert np.array_equal(X @ inst.A.T.astype(np.int64), np.tile(inst.d, (len(X), 1)))
        assert any(np.array_equal(inst.planted, x) for x in st.solutions)
        keys = ["".join(map(str, x)) for x in st.solutions]
        assert keys == sorted(set(keys))
        assert st.leaves >= len(X) and st.passed >= st.leaves and st.nodes >= st.passed
