"""The paper's larger configurations at full size, in the launch configuration
of `bench.py --workload m8_all | m9_all` (BKZ-10, automatic lanes).

m = 8, n = 70, D = 200 (16 instances): every instance's node count and
solution set equal the oracle's (the oracle runs in a process pool started
with spawn, before any GPU work).  m = 9, n = 80, D = 100 (8 instances): the
oracle needs about an hour per instance, so its complete results are stored
in tests/golden/m9_n80_d100_bkz10.txt (written by the script beside it, which
calls only the oracle); the GPU's solution sets, node counts and reduced
bases must equal them, and sampled subtrees are also re-enumerated by the
oracle here."""
import multiprocessing as mp

import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_08702_gb300 import instances as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _oracle_job(args):
    A, d, lanes = args
    _, kern, _ = O.reduce(A, d)
    kb = O.bkz(kern, 10).kern
    r = O.enumerate(kb, O.gso(kb), A, d, lanes=lanes)
    return r.nodes, r.solutions


@pytest.fixture(scope="module")
def m8_oracle():
    insts = I.m8_n70(16)
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, mp.cpu_count())) as pool:
        async_res = pool.map_async(_oracle_job, [(x.A, x.d, 16) for x in insts])
        yield insts, async_res
        async_res.wait()


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


def test_m8_all_solutions_equal_oracle(m8_oracle):
    insts, async_res = m8_oracle
    res, sols, ctx = M().solve(insts, bkz_beta=10, max_seconds=300.0)
    assert ctx.lanes == 16
    ref = async_res.get(timeout=1200)
    for i, inst in enumerate(insts):
        assert res.stats[i]["status"] == 0
        assert res.stats[i]["nodes"] == ref[i][0], i
        assert np.array_equal(sols[i], ref[i][1]), i
        assert any(np.array_equal(inst.planted, x) for x in sols[i]), i
    ctx.close()


@pytest.fixture(scope="module")
def m9_gpu():
    insts = I.m9_n80(8)
    res, sols, ctx = M().solve(insts, bkz_beta=10, max_seconds=900.0)
    yield insts, res, sols, ctx
    ctx.close()


def test_m9_all_solutions_equal_the_stored_oracle_results(m9_gpu):
    from tests.golden import m9_golden
    gold = m9_golden.load()
    insts, res, sols, ctx = m9_gpu
    assert ctx.lanes == gold.lanes
    for i, inst in enumerate(insts):
        g = gold.instances[inst.seed]
        assert res.stats[i]["status"] == 0
        assert m9_golden.basis_digest(ctx.msp_export_gso(i)[0]) == g.digest, i
        st = res.stats[i]
        assert (st["nodes"], st["passed"], st["leaves"]) == (g.nodes, g.passed, g.leaves), i
        assert np.array_equal(sols[i], g.solutions), i


def test_m9_all_solutions_on_sampled_subtrees(m9_gpu):
    insts, res, sols, ctx = m9_gpu
    rng = np.random.default_rng(9)
    for i, inst in enumerate(insts):
        assert res.stats[i]["status"] == 0
        for x in sols[i].astype(np.int64):
            assert np.array_equal(inst.A.astype(np.int64) @ x, inst.d)
        assert any(np.array_equal(inst.planted, x) for x in sols[i]), i
        # the GPU's reduced basis is the oracle's (bit-exact), so its subtrees are too
        _, kern, _ = O.reduce(inst.A, inst.d)
        kb = O.bkz(kern, 10).kern
        assert np.array_equal(ctx.msp_export_gso(i)[0], kb), i
        g = O.gso(kb)
        p = ctx.msp_export_prefixes(i)
        small = np.argsort(p["nodes"])[: max(1, len(p["nodes"]) // 4)]   # oracle-sized subtrees
        for j in rng.choice(small, size=min(3, len(small)), replace=False):
            sub = O.enumerate(kb, g, inst.A, inst.d, lanes=ctx.lanes, sub_level=p["split_level"] - 1,
                              prefix=p["u"][j])
            assert sub.nodes == p["nodes"][j], (i, j)
            assert len(sub.solutions) == p["sols"][j], (i, j)
