"""GPU parity for the general problem of Sec. 2 (bounds 0 <= x_j <= r_j)
against the oracle: node counts exact, solution sets equal (and equal to
brute force over the box where it is small), binary instances in the same
batch unchanged."""
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


BOUNDED = [I.bounded(700 + s, *a) for s in range(2) for a in
           [(2, 14, 40, (1, 2, 3)), (3, 18, 30, (1, 2, 3)), (2, 12, 60, (4, 5, 6)), (3, 20, 40, (1, 2)),
            (4, 24, 30, (1, 2)), (2, 10, 50, (1, 2, 3, 4, 5, 6, 7)), (5, 36, 50, (1, 2)),
            (4, 30, 60, (1, 2, 3)), (3, 16, 40, (1, 2, 3, 4, 5, 6, 7))]]


def M():
    from paper_2508_08702_gb300 import msp
    return msp


def _check(insts, res, sols, **kw):
    for i, inst in enumerate(insts):
        ref = O.solve(inst.A, inst.d, r=inst.r, lanes=8, **kw).result
        st = res.stats[i]
        assert (st["nodes"], st["passed"], st["leaves"]) == (ref.nodes, ref.passed, ref.leaves), (i, inst.tag)
        assert np.array_equal(sols[i], ref.solutions), (i, inst.tag)
        assert any(np.array_equal(inst.planted, x) for x in sols[i]), i
        if inst.r is not None and np.prod(inst.r.astype(float) + 1) <= 1 << 20:
            assert np.array_equal(sols[i], DEF.brute_force_bounds(inst.A, inst.d, inst.r)), i


@pytest.mark.parametrize("depth", [0, 6, 24])
def test_bounded_batch_equals_oracle(depth):
    res, sols, ctx = M().solve(BOUNDED, lanes=8, split_depth=depth, max_seconds=120.0)
    _check(BOUNDED, res, sols)
    ctx.close()


@pytest.mark.parametrize("hoelder,sym", [(0, 0), (1, 1), (2, 1)])
def test_bounded_pruning_modes(hoelder, sym):
    insts = BOUNDED[:6]
    res, sols, ctx = M().solve(insts, lanes=8, hoelder=hoelder, sym=sym, max_seconds=120.0)
    _check(insts, res, sols, hoelder={0: O.HOELDER_CUT, 1: O.HOELDER_FILTER, 2: O.HOELDER_OFF}[hoelder],
           sym=bool(sym))
    ctx.close()


def test_mixed_batch_keeps_binary_results():
    binary = [I.small(1000 + s, 3, 20, 8) for s in range(3)]
    insts = binary[:2] + BOUNDED[:3] + binary[2:]
    res, sols, ctx = M().solve(insts, lanes=8, max_seconds=120.0)
    for i, inst in enumerate(insts):
        ref = O.solve(inst.A, inst.d, r=inst.r, lanes=8).result
        assert res.stats[i]["nodes"] == ref.nodes, i
        assert np.array_equal(sols[i], ref.solutions), i
    ctx.close()


def test_binary_without_slack_equals_oracle():
    """use_eps = 0: the integer filter must carry no slack either."""
    insts = [I.small(1000 + s, m, n, D) for s in range(2) for (m, n, D) in [(2, 18, 12), (3, 20, 8)]]
    res, sols, ctx = M().solve(insts, lanes=8, use_eps=0, max_seconds=120.0)
    for i, inst in enumerate(insts):
        ref = O.solve(inst.A, inst.d, lanes=8, use_eps=False).result
        assert res.stats[i]["nodes"] == ref.nodes, i
        assert np.array_equal(sols[i], ref.solutions), i
    ctx.close()


def test_bound_limits_are_rejected():
    inst = BOUNDED[0]
    ctx = M().Context()
    pk = I.pack([inst])
    for bad in (np.zeros(inst.n, np.int32), np.full(inst.n, 256, np.int32)):
        with pytest.raises(M().MspError):
            ctx.msp_build_lattice(pk.dims, pk.A, pk.d, bad)
    r = np.ones(inst.n, np.int32)
    r[:4] = [7, 11, 13, 17]          # lcm 17017 > 1024
    with pytest.raises(M().MspError):
        ctx.msp_build_lattice(pk.dims, pk.A, pk.d, r)
    big = I.small(1, 2, 60, 10)      # 60 variables x 3 bits > 128
    with pytest.raises(M().MspError):
        ctx.msp_build_lattice(I.pack([big]).dims, big.A, big.d, np.full(60, 4, np.int32))
    ctx.close()
