"""CUDA graph replay of a whole step, and the autotuner, on the GPU."""
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


def _per_instance(ctx, res):
    return [(s["nodes"], s["solutions"]) for s in res.stats], [ctx.msp_solutions(i) for i in range(ctx.count)]


def test_graph_replay_equals_eager_step():
    from paper_2508_08702_gb300 import msp as M
    insts = I.batch_m4_7(12)
    pk = I.pack(insts)
    ctx = M.Context(max_seconds=120.0)
    ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
    ctx.msp_run_async()
    eager, eager_x = _per_instance(ctx, ctx.msp_wait())
    ctx.msp_graph_capture()
    for _ in range(2):
        ctx.msp_graph_launch()
        got, got_x = _per_instance(ctx, ctx.msp_wait())
        assert got == eager
        for a, b in zip(got_x, eager_x):
            assert np.array_equal(a, b)
        ph = ctx.msp_phase_ms()
        assert ph["enumerate"] > 0 and ph["reduce"] > 0
    ctx.close()


def test_graph_replay_on_new_batch_of_same_layout():
    """New A, d with the same (m, n) per instance: the captured graph solves
    the new batch; nodes equal the oracle's."""
    from paper_2508_08702_gb300 import msp as M
    first = [I.small(7000 + s, 3, 20, 10) for s in range(4)]
    second = [I.small(7100 + s, 3, 20, 10) for s in range(4)]
    ctx = M.Context(max_seconds=120.0, lanes=8)
    pk = I.pack(first)
    ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
    ctx.msp_run_async()
    ctx.msp_wait()
    ctx.msp_graph_capture()
    pk2 = I.pack(second)
    ctx.msp_build_lattice(pk2.dims, pk2.A, pk2.d)
    ctx.msp_graph_launch()
    res = ctx.msp_wait()
    for i, inst in enumerate(second):
        ref = O.solve(inst.A, inst.d, lanes=8).result
        assert res.stats[i]["nodes"] == ref.nodes
        assert np.array_equal(ctx.msp_solutions(i), ref.solutions)
    # a different layout discards the graph
    pk3 = I.pack(second[:3])
    ctx.msp_build_lattice(pk3.dims, pk3.A, pk3.d)
    with pytest.raises(M.MspError):
        ctx.msp_graph_launch()
    ctx.close()


def test_graph_capture_requires_a_completed_step():
    from paper_2508_08702_gb300 import msp as M
    pk = I.pack(I.single_m3())
    ctx = M.Context()
    ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
    with pytest.raises(M.MspError):
        ctx.msp_graph_capture()
    with pytest.raises(M.MspError):
        ctx.msp_graph_launch()
    ctx.close()


def test_tuner_picks_a_working_shape():
    from paper_2508_08702_gb300 import tune
    insts = I.batch_m4_7(8)
    out = tune.tune(insts, grid={"lanes": (8, 16), "split_target": (0,)})
    assert np.isfinite(out["ms"]) and out["ms"] > 0
    assert out["opts"]["lanes"] in (8, 16)
    assert len(out["table"]) == 2
