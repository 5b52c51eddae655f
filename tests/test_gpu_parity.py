"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer results (reduced bases, solution sets, node counts) must match
bit for bit; the FP64 Gram-Schmidt tables too, since both sides perform the
same IEEE operations in the same order.  Sizes span several tiles (lane
groups, walkers, split levels) with ragged tails; the full-size batch of the
benchmark is checked on properties and on sampled subtrees.
"""
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


def msp():
    from paper_2508_08702_gb300 import msp as M
    return M


SMALL = [I.small(1000 + s, m, n, D)
         for s in range(3)
         for (m, n, D) in [(1, 16, 60), (2, 18, 12), (3, 20, 8), (2, 20, 30), (4, 22, 6), (3, 21, 100)]]
HMODE = {0: O.HOELDER_CUT, 1: O.HOELDER_FILTER, 2: O.HOELDER_OFF}


def run_gpu(instances, **opts):
    M = msp()
    opts.setdefault("max_seconds", 120.0)
    res, sols, ctx = M.solve(instances, **opts)
    return res, sols, ctx


def test_reduction_and_tables_bit_exact():
    """LLL basis, kernel basis and FP64 tables equal the oracle's exactly."""
    insts = I.single_m3() + SMALL[:6] + I.batch_m4_7(6)
    M = msp()
    pk = I.pack(insts)
    ctx = M.Context()
    ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
    ctx.msp_reduce()
    for i, inst in enumerate(insts):
        red = O.lll(O.build_lattice(inst.A, inst.d))
        assert np.array_equal(ctx.msp_export_reduced(i), red.basis), i
        kern = O.extract(red.basis, inst.m)
        g = O.gso(kern)
        kb, mu, B, bhat = ctx.msp_export_gso(i)
        assert np.array_equal(kb, kern), i
        assert np.array_equal(B, g.B), i
        assert np.array_equal(np.tril(mu), np.tril(g.mu)), i
        assert np.array_equal(bhat, g.bhat), i
    ctx.close()


@pytest.mark.parametrize("lanes", [8, 16, 32])
def test_small_batch_solutions_and_nodes(lanes):
    """One launch over 18 small instances: solution sets equal brute force,
    node counts equal the oracle's (same l1 summation order)."""
    res, sols, ctx = run_gpu(SMALL, lanes=lanes)
    for i, inst in enumerate(SMALL):
        want = DEF.brute_force(inst.A, inst.d)
        assert np.array_equal(sols[i], want), i
        ref = O.solve(inst.A, inst.d, lanes=lanes).result
        st = res.stats[i]
        assert (st["nodes"], st["passed"], st["leaves"]) == (ref.nodes, ref.passed, ref.leaves), i
    ctx.close()


@pytest.mark.parametrize("hoelder", [0, 1, 2])
@pytest.mark.parametrize("sym", [1, 0])
def test_pruning_modes(hoelder, sym):
    insts = SMALL[:6]
    res, sols, ctx = run_gpu(insts, hoelder=hoelder, sym=sym, lanes=16)
    for i, inst in enumerate(insts):
        ref = O.solve(inst.A, inst.d, hoelder=HMODE[hoelder], sym=bool(sym), lanes=16).result
        assert np.array_equal(sols[i], ref.solutions)
        assert res.stats[i]["nodes"] == ref.nodes
    ctx.close()


@pytest.mark.parametrize("depth", [0, 1, 4, 12, 24])
def test_split_depth_invariance(depth):
    """Node totals and solutions do not depend on how deep the splitter goes."""
    insts = [x for x in I.batch_m4_7(16) if x.m <= 6]   # depth 0 = one walker per tree
    res, sols, ctx = run_gpu(insts, split_depth=depth, lanes=16)
    for i, inst in enumerate(insts):
        ref = O.solve(inst.A, inst.d, lanes=16).result
        assert np.array_equal(sols[i], ref.solutions), i
        assert res.stats[i]["nodes"] == ref.nodes, (i, depth)
    ctx.close()


def test_splitter_prefixes_equal_oracle_split():
    insts = I.batch_m4_7(8)
    res, sols, ctx = run_gpu(insts, lanes=16)
    for i, inst in enumerate(insts):
        p = ctx.msp_export_prefixes(i)
        _, kern, g = O.reduce(inst.A, inst.d)
        ref = O.enumerate(kern, g, inst.A, inst.d, lanes=16, split_level=p["split_level"])
        assert np.array_equal(p["u"][:, p["split_level"]:], ref.prefixes[:, p["split_level"]:]), i
        assert np.array_equal(p["rho"], ref.prefix_rho), i
        # the subtree log adds up with the split part to the instance total
        assert p["nodes"].sum() + ref.nodes == res.stats[i]["nodes"], i
    ctx.close()


def test_full_batch_in_bench_configuration():
    """The 64-instance batch exactly as the benchmark launches it: every
    reported x is binary with A x = d, every planted x is found, solution
    sets equal the oracle where it is fast, and a sample of subtrees of the
    large instances matches the oracle node for node."""
    insts = I.batch_m4_7(64)
    res, sols, ctx = run_gpu(insts)
    lanes = ctx.lanes
    rng = np.random.default_rng(0)
    for i, inst in enumerate(insts):
        x = sols[i].astype(np.int64)
        assert res.stats[i]["status"] == 0
        assert len(x) == res.stats[i]["solutions"] > 0
        assert np.all(x @ inst.A.T.astype(np.int64) == inst.d[None, :])
        assert any(np.array_equal(inst.planted, s) for s in sols[i])
        assert len({bytes(s) for s in sols[i]}) == len(sols[i])
        if inst.m <= 5:
            assert np.array_equal(sols[i], DEF.meet_in_middle(inst.A, inst.d))
        if inst.m <= 6:
            ref = O.solve(inst.A, inst.d, lanes=lanes).result
            assert res.stats[i]["nodes"] == ref.nodes
        elif i % 4 == 0:
            p = ctx.msp_export_prefixes(i)
            _, kern, g = O.reduce(inst.A, inst.d)
            pick = rng.choice(len(p["u"]), size=min(6, len(p["u"])), replace=False)
            for j in pick:
                sub = O.enumerate(kern, g, inst.A, inst.d, lanes=lanes,
                                  sub_level=p["split_level"] - 1, prefix=p["u"][j])
                assert sub.nodes == p["nodes"][j], (i, j)
                assert len(sub.solutions) == p["sols"][j], (i, j)
    ctx.close()


def test_first_mode_stops_with_a_valid_solution():
    M = msp()
    insts = I.batch_m4_7(4)
    res, sols, ctx = run_gpu(insts, mode=M.MSP_FIRST)
    found = [i for i in range(len(insts)) if len(sols[i])]
    assert found
    for i in found:
        x = sols[i].astype(np.int64)
        assert np.all(x @ insts[i].A.T.astype(np.int64) == insts[i].d[None, :])
    ctx.close()


def test_time_cap_returns_partial_results():
    M = msp()
    inst = I.batch_m4_7(4)[3]   # m=7, D=50: about 2.6e8 nodes
    assert inst.m == 7
    res, sols, ctx = run_gpu([inst], time_cap_s=0.02, allow=(M.MSP_OK, M.MSP_ETIMEOUT))
    assert res.status in (M.MSP_OK, M.MSP_ETIMEOUT)
    for x in sols[0].astype(np.int64):
        assert np.array_equal(x @ inst.A.T.astype(np.int64), inst.d)
    ctx.close()


def test_edge_cases():
    """Single-column, single-level and infeasible instances; ragged batch."""
    rng = np.random.default_rng(3)
    cases = []
    A = np.array([[7]], np.int32)
    cases.append((A, np.array([7], np.int64)))          # n = 1: x = 1
    cases.append((A, np.array([0], np.int64)))          # n = 1: x = 0
    A2 = 2 * rng.integers(0, 30, size=(2, 18)).astype(np.int32)
    cases.append((A2, ((A2.sum(axis=1) // 2) | 1).astype(np.int64)))   # infeasible (parity)
    A3 = rng.integers(0, 5, size=(1, 12)).astype(np.int32)
    cases.append((A3, np.array([A3.sum() // 2], np.int64)))             # many solutions
    A4 = rng.integers(0, 1000, size=(6, 6)).astype(np.int32)            # m = n
    cases.append((A4, A4.astype(np.int64) @ np.array([1, 0, 1, 1, 0, 1])))

    class X:
        def __init__(self, A, d):
            self.A, self.d = A, d
            self.m, self.n = A.shape
    insts = [X(a, d) for a, d in cases]
    res, sols, ctx = run_gpu(insts)
    for i, x in enumerate(insts):
        want = DEF.brute_force(x.A, x.d)
        assert np.array_equal(sols[i], want), i
        ref = O.solve(x.A, x.d, lanes=ctx.lanes).result
        assert res.stats[i]["nodes"] == ref.nodes, i
    ctx.close()


def test_argument_errors_and_call_order():
    M = msp()
    with pytest.raises(M.MspError) as e:
        M.Context(lanes=12)
    assert e.value.status == M.MSP_EINVAL
    ctx = M.Context()
    with pytest.raises(M.MspError) as e:
        ctx.msp_reduce()
    assert e.value.status == M.MSP_ESTATE
    with pytest.raises(M.MspError) as e:
        ctx.msp_build_lattice(np.array([[3, 2]]), np.zeros(6, np.int32), np.zeros(3, np.int64))
    assert e.value.status == M.MSP_EINVAL     # m > n
    with pytest.raises(M.MspError) as e:
        ctx.msp_build_lattice(np.array([[1, 200]]), np.zeros(200, np.int32), np.zeros(1, np.int64))
    assert e.value.status == M.MSP_EINVAL     # n + 1 > 128
    ctx.close()


def test_device_resident_inputs_match_host_inputs():
    M = msp()
    insts = I.batch_m4_7(8)
    pk = I.pack(insts)
    ctx = M.Context()
    ctx.msp_build_lattice(pk.dims, torch.from_numpy(pk.A).cuda(), torch.from_numpy(pk.d).cuda())
    ctx.msp_run_async()
    r1 = ctx.msp_wait()
    s1 = [ctx.msp_solutions(i) for i in range(len(insts))]
    ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
    ctx.msp_reduce()
    r2 = ctx.msp_enumerate()
    for i in range(len(insts)):
        assert r1.stats[i]["nodes"] == r2.stats[i]["nodes"]
        assert np.array_equal(s1[i], ctx.msp_solutions(i))
    ctx.close()


def test_too_small_scale_is_reported():
    """With N = 1 the reduction cannot isolate the kernel lattice (Sec. 2
    needs N large); the library reports MSP_ERANK instead of enumerating an
    incomplete basis."""
    M = msp()
    insts = I.batch_m4_7(3)
    res, sols, ctx = run_gpu(insts, N=1, allow=(M.MSP_ERANK,))
    assert res.status == M.MSP_ERANK
    assert all(s["status"] == M.MSP_ERANK for s in res.stats)
    ctx.close()


WIDE = [I.make_instance(6000 + m + n, m, n, D, tag=f"wide_m{m}n{n}")
        for (m, n, D) in [(20, 70, 100), (16, 70, 100), (24, 90, 100), (28, 100, 50)]]


@pytest.mark.parametrize("lanes", [4, 8, 16, 32])
def test_every_lane_count_on_every_width(lanes):
    """Lattice widths n+1 from 21 to 101 (row padding 32, 64, 96, 128) under
    every lane count: node counts and solutions equal the oracle's."""
    insts = WIDE + [x for x in I.batch_m4_7(8) if x.m <= 5] + SMALL[:3]
    res, sols, ctx = run_gpu(insts, lanes=lanes)
    for i, inst in enumerate(insts):
        ref = O.solve(inst.A, inst.d, lanes=lanes).result
        assert np.array_equal(sols[i], ref.solutions), (i, inst.tag)
        assert res.stats[i]["nodes"] == ref.nodes, (i, inst.tag)
    ctx.close()


MAXI = [I.make_instance(7100, 32, 127, 50, tag="max_m32n127"),     # the most rows, the widest lattice
        I.make_instance(7102, 24, 127, 100, tag="max_m24n127"),
        I.make_instance(7200, 6, 127, 100, tag="max_m6n127")]       # 58 solutions within budget 4


@pytest.mark.parametrize("lanes", [8, 16])
def test_maximum_sizes(lanes):
    """n + 1 = 128 lattice coordinates and m = 32 rows, the largest the
    library accepts: LLL and kernel bases and FP64 tables bit-exact, the
    split prefixes exact, one discrepancy iteration of budget 4 (10^6 to
    10^7 nodes) node- and set-exact; one row or one column more is
    rejected with MSP_EINVAL."""
    M = msp()
    res, sols, ctx = run_gpu(MAXI, order=M.MSP_LDS, lds_budget=4, lanes=lanes)
    found = 0
    for i, inst in enumerate(MAXI):
        red = O.lll(O.build_lattice(inst.A, inst.d))
        assert np.array_equal(ctx.msp_export_reduced(i), red.basis), i
        kern = O.extract(red.basis, inst.m)
        g = O.gso(kern)
        kb, mu, B, bhat = ctx.msp_export_gso(i)
        assert kb.shape[1] == 128
        assert np.array_equal(kb, kern), i
        assert np.array_equal(B, g.B), i
        assert np.array_equal(np.tril(mu), np.tril(g.mu)), i
        assert np.array_equal(bhat, g.bhat), i
        ref = O.enumerate(kern, g, inst.A, inst.d, lanes=lanes, lds=4)
        st = res.stats[i]
        assert (st["nodes"], st["passed"], st["leaves"]) == (ref.nodes, ref.passed, ref.leaves), (i, lanes)
        assert np.array_equal(sols[i], ref.solutions), i
        found += len(ref.solutions)
        p = ctx.msp_export_prefixes(i)
        lvl = p["split_level"]
        top = O.enumerate(kern, g, inst.A, inst.d, lanes=lanes, split_level=lvl, lds=4)   # budgeted top levels
        assert np.array_equal(p["u"][:, lvl:], top.prefixes[:, lvl:]), i
        assert np.array_equal(p["rho"], top.prefix_rho), i
    assert found > 0
    ctx.close()
    ctx = M.Context()
    for m, n in [(1, 128), (33, 40)]:
        with pytest.raises(M.MspError) as e:
            ctx.msp_build_lattice(np.array([[m, n]]), np.zeros(m * n, np.int32), np.zeros(m, np.int64))
        assert e.value.status == M.MSP_EINVAL, (m, n)
    ctx.close()
