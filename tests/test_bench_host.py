"""Host-side logic of the benchmark (no GPU): the table of paper-shaped
workloads, the oracle baseline's sample, the roofline's operation count and
the one-instance-per-core oracle leg."""
import numpy as np
import pytest

import bench
from paper_2508_08702_gb300 import instances as I


def _instances(gen):
    return bench.make_instances(gen)


@pytest.mark.parametrize("name", sorted(bench.WORKLOADS))
def test_workloads_have_the_paper_shapes(name):
    """Sec. 4 / Table 1 shapes: n = 10(m-1), a_ij in [0, D), d = A x for the
    planted x; the generators are deterministic."""
    gen, mode, cap = bench.WORKLOADS[name]
    assert mode in ("all", "first") and cap > 0
    xs = _instances(gen)
    assert xs
    for x in xs:
        assert x.n == 10 * (x.m - 1)
        assert x.A.shape == (x.m, x.n)
        assert x.A.min() >= 0 and x.A.max() < x.D
        if x.planted is not None:
            assert np.array_equal(x.A.astype(np.int64) @ x.planted.astype(np.int64), x.d)
    again = _instances(gen)
    assert all(np.array_equal(a.A, b.A) and np.array_equal(a.d, b.d) for a, b in zip(xs, again))


def test_evaluation_seeds_are_disjoint_from_the_training_set():
    train = {x.seed for x in I.training_set(256)}
    evals = {x.seed for x in I.batch_m4_7(64)}
    for gen, _, _ in bench.WORKLOADS.values():
        evals |= {x.seed for x in _instances(gen)}
    assert not train & evals


def test_baseline_sample_keeps_batch_order():
    batch = I.batch_m4_7(64)
    sample = bench.cpu_baseline_sample(batch)
    assert [x.tag for x in sample] == [x.tag for x in batch if x.m <= 6 or (x.m == 7 and x.D >= 100)]
    assert any(x.m == 7 for x in sample)
    assert [x.tag for x in bench.cpu_sample(batch)] == [x.tag for x in batch if x.m <= 6]


def test_oracle_rate_repeats_passes_to_the_minimum_time():
    xs = [I.small(7200 + i, 3, 12, 20) for i in range(2)]
    v, nodes, dt, runs = bench.oracle_nodes_per_s(xs, 60.0, lanes=8, min_seconds=0.2)
    assert dt >= 0.2 and runs >= 2 and runs % 1 == 0
    assert nodes > 0 and v == pytest.approx(nodes / dt)


def test_headline_workloads_are_the_m12_rows():
    for key, gen, runs, desc in bench.HEADLINE_FIRST:
        xs = bench.make_instances(gen)
        for orders, cap, extra in runs:
            assert cap > 0 and set(orders.split(",")) <= {"plain", "learned", "lds", "lds_learned"}
        assert len(xs) == 4 and all(x.m == 12 and x.n == 110 for x in xs)
        assert f"D={xs[0].D}" in desc


def test_algorithmic_operation_count():
    """3 per evaluated node past the split, 2(n+1) + log2 G + 1 per node that
    passes the norm test above level 0, plus the centre-fold fmas."""
    stats = [{"nodes": 1000, "split_nodes": 100, "passed": 600, "split_passed": 50, "leaves": 20,
              "center_fma": 7},
             {"nodes": 10, "split_nodes": 0, "passed": 4, "split_passed": 0, "leaves": 4, "center_fma": 0}]
    dims = [(5, 40), (3, 20)]
    assert bench.algorithmic_fp64_ops(stats, dims, 8) == 3 * 900 + (82 + 3 + 1) * 530 + 7 + 3 * 10
    assert bench.algorithmic_fp64_ops(stats[:1], dims[:1], 16) == 3 * 900 + (82 + 4 + 1) * 530 + 7


def test_host_cpu_reports_the_cores():
    h = bench.host_cpu()
    assert h["nproc"] >= 1 and h["machine"]


def test_parallel_oracle_leg_counts_the_same_nodes():
    from oracle import oracle as O
    xs = [I.small(7100 + i, 3, 14, 20) for i in range(3)]
    want = sum(O.solve(x.A, x.d).result.nodes for x in xs)
    value, nodes, seconds = bench.oracle_parallel_nodes_per_s(xs, 2)
    assert nodes == want
    assert value > 0 and seconds > 0
