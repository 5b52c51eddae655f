"""The fused launch (msp_opts.fuse, an option of msp_run_async and graph
capture for all-solutions depth-first steps): the blocks of the enumeration
kernel reduce and split the instances themselves and publish each one's
subtrees as they finish.  It runs the same device functions as the separate
launches, so every reduced basis, node count and solution set must be equal
to theirs, and to the oracle's."""
import numpy as np
import pytest

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


def M():
    from paper_2508_08702_gb300 import msp
    return msp


def _step(insts, fuse, **kw):
    pk = I.pack(insts)
    ctx = M().Context(fuse=fuse, max_seconds=30.0, **kw)
    ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
    ctx.msp_run_async()
    res = ctx.msp_wait()
    sols = [ctx.msp_solutions(i) for i in range(len(insts))]
    bases = [ctx.msp_export_gso(i)[0] for i in range(ctx.count)]
    launches = ctx.kernel_launches
    ctx.close()
    return res, sols, bases, launches


@pytest.mark.parametrize("kw", [{}, {"bkz_beta": 10}, {"lanes": 16}, {"split_target": 64},
                                {"warps_per_block": 4}], ids=["default", "bkz10", "lanes16", "split64", "warps4"])
def test_fused_step_equals_separate_launches(kw):
    insts = I.batch_m4_7(24)
    r0, s0, b0, n0 = _step(insts, 0, **kw)
    r1, s1, b1, n1 = _step(insts, 1, **kw)
    assert n1 < n0   # the reduction and split launches are gone
    for i in range(len(insts)):
        a, b = r0.stats[i], r1.stats[i]
        for key in ("status", "nodes", "passed", "leaves", "solutions", "kernel_rank", "lll_iterations",
                    "lll_swaps", "bkz_tours", "bkz_inserts", "prefixes", "split_nodes"):
            assert a[key] == b[key], (i, key, a[key], b[key])
        assert np.array_equal(s0[i], s1[i]), i
        assert np.array_equal(b0[i], b1[i]), i


def test_fused_step_equals_the_oracle():
    insts = [x for x in I.batch_m4_7(16) if x.m <= 6]
    res, sols, bases, _ = _step(insts, 1, lanes=8)
    for i, inst in enumerate(insts):
        ref = O.solve(inst.A, inst.d, lanes=8).result
        assert res.stats[i]["nodes"] == ref.nodes, i
        assert np.array_equal(sols[i], ref.solutions), i


def test_fused_step_with_replicas_and_failed_instances():
    """Replicas shuffle the columns before the fused launch; an instance whose
    reduction fails publishes no subtrees and the others still finish."""
    insts = I.batch_m4_7(6)
    r0, s0, _, _ = _step(insts, 0, replicas=3)
    r1, s1, _, _ = _step(insts, 1, replicas=3)
    for i in range(len(insts)):
        assert r0.stats[i]["nodes"] == r1.stats[i]["nodes"], i
        assert np.array_equal(s0[i], s1[i]), i
    # an LLL iteration cap of 1 stops every reduction: nothing to enumerate
    pk = I.pack(insts)
    ctx = M().Context(fuse=1, lll_max_iter=1, max_seconds=60.0)
    ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
    ctx.msp_run_async()
    res = ctx.msp_wait(allow=(M().MSP_OK, M().MSP_ECAP))
    assert all(s["status"] == M().MSP_ECAP for s in res.stats)
    assert res.total["nodes"] == 0
    ctx.close()


def test_fused_graph_replay_equals_a_fresh_step():
    insts = I.batch_m4_7(12)
    pk = I.pack(insts)
    r0, s0, _, _ = _step(insts, 1)
    ctx = M().Context(fuse=1, max_seconds=30.0)
    ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
    ctx.msp_run_async()
    ctx.msp_wait()
    ctx.msp_graph_capture()
    for _ in range(2):
        ctx.msp_graph_launch()
        res = ctx.msp_wait()
        for i in range(len(insts)):
            assert res.stats[i]["nodes"] == r0.stats[i]["nodes"], i
            assert np.array_equal(ctx.msp_solutions(i), s0[i]), i
    ctx.close()
