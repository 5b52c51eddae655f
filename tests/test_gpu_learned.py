"""GPU tests of the subtree scorer and the queue orders.

The tensor-core kernels are compared with oracle/mlp.py (same bfloat16
roundings of inputs, weights and activations; float32 vs float64 sums and
the kernels' bfloat16 rounding of the back-propagated gradients make up the
tolerances written below).  The learned order must leave the all-solutions
results unchanged node for node."""
import numpy as np
import pytest

from oracle import mlp as R
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


def M():
    from paper_2508_08702_gb300 import msp
    return msp


def test_mlp_forward_matches_reference():
    rng = np.random.default_rng(0)
    theta = R.init(1)
    theta[2048:2112] = rng.normal(0, 0.2, 64)          # nonzero biases
    x = rng.normal(0, 1, size=(1037, 32)).astype(np.float32)   # ragged tail of 13 rows
    ctx = M().Context()
    y = torch.zeros((len(x), 8), dtype=torch.float32, device="cuda")
    ctx.msp_mlp_forward(torch.from_numpy(theta).cuda(), torch.from_numpy(x).cuda(), y)
    got = y.cpu().numpy()
    want, _ = R.forward(theta, x)
    err = np.abs(got - want)
    assert np.median(err) < 1e-4
    # a float32 sum landing on the other side of a bfloat16 rounding boundary
    # can move one activation by 2^-8 of its size
    assert np.all(err <= 2e-2 * (1 + np.abs(want)))
    ctx.close()


@pytest.mark.parametrize("n", [128, 300, 1037])
def test_mlp_gradient_matches_reference(n):
    """Every gradient element, block by block (W1, b1, W2, b2, W3, b3),
    against the oracle evaluated with the kernels' precision contract
    (bfloat16 operands at the stated rounding points, float64 sums); the
    tolerances and why they hold are in tests/mlp_check.py."""
    from tests.mlp_check import block_failures
    rng = np.random.default_rng(n)
    theta = R.init(2) * 0.8
    theta[2048:2112] = rng.normal(0, 0.1, 64)          # nonzero b1
    theta[6208:6272] = rng.normal(0, 0.1, 64)          # nonzero b2
    theta[6784:6792] = rng.normal(0, 0.1, 8)           # nonzero b3
    x = rng.normal(0, 1, size=(n, 32)).astype(np.float32)
    found = (rng.random(n) < 0.2).astype(np.float32)
    ln = rng.normal(4, 1, n).astype(np.float32)
    target = np.stack([found, ln], axis=1).astype(np.float32)
    ctx = M().Context()
    g = torch.zeros(R.MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ctx.msp_mlp_grad(torch.from_numpy(theta).cuda(), torch.from_numpy(x).cuda(), torch.from_numpy(target).cuda(),
                     3.0, g, loss)
    want_loss, want, scale = R.loss_and_grad(theta, x, found, ln, 3.0, round_grad_bf16=True, scales=True)
    got = g.cpu().numpy().astype(np.float64)
    assert float(loss.cpu()) == pytest.approx(want_loss, rel=1e-4)
    assert block_failures(got, want, scale, R.blocks) == []
    ctx.close()


def test_mlp_training_reduces_loss():
    rng = np.random.default_rng(7)
    n = 4096
    x = rng.normal(0, 1, size=(n, 32)).astype(np.float32)
    found = ((x[:, 0] + 0.5 * x[:, 1]) > 1.2).astype(np.float32)
    ln = (3.0 + x[:, 2] - 0.5 * x[:, 3]).astype(np.float32)
    target = np.stack([found, ln], axis=1)
    theta = torch.from_numpy(R.init(3)).cuda()
    losses = torch.zeros(600, dtype=torch.float32, device="cuda")
    ctx = M().Context()
    ctx.msp_mlp_train(theta, torch.from_numpy(x).cuda(), torch.from_numpy(target).cuda(), 600, 3e-3, 1.0, 11,
                      losses)
    L = losses.cpu().numpy()
    assert np.all(np.isfinite(L))
    assert L[-50:].mean() < 0.3 * L[:20].mean()
    # the trained network separates the classes on fresh data
    xt = rng.normal(0, 1, size=(2000, 32)).astype(np.float32)
    yt = torch.zeros((2000, 8), dtype=torch.float32, device="cuda")
    ctx.msp_mlp_forward(theta, torch.from_numpy(xt).cuda(), yt)
    pred = yt.cpu().numpy()[:, 0] > 0
    truth = (xt[:, 0] + 0.5 * xt[:, 1]) > 1.2
    assert (pred == truth).mean() > 0.93
    ctx.close()


def test_learned_order_keeps_all_mode_exact():
    """The order only decides when a subtree is walked, never which nodes."""
    insts = [x for x in I.batch_m4_7(20) if x.m <= 6]
    theta = R.init(9)
    msp = M()
    r_plain, s_plain, c1 = msp.solve(insts, max_seconds=120.0)
    r_learn, s_learn, c2 = msp.solve(insts, order=msp.MSP_LEARNED, scorer=theta, max_seconds=120.0)
    for i, inst in enumerate(insts):
        assert r_learn.stats[i]["nodes"] == r_plain.stats[i]["nodes"]
        assert np.array_equal(s_learn[i], s_plain[i])
        ref = O.solve(inst.A, inst.d, lanes=c1.lanes).result
        assert r_learn.stats[i]["nodes"] == ref.nodes
    c1.close()
    c2.close()


@pytest.mark.parametrize("learned", [False, True])
def test_first_mode_stops_each_instance_on_a_valid_solution(learned):
    from paper_2508_08702_gb300 import learn
    insts = I.batch_m4_7(12)
    msp = M()
    run = learn.first_solution(insts, msp.MSP_LEARNED if learned else msp.MSP_PLAIN,
                               scorer=R.init(4) if learned else None, max_seconds=120.0)
    assert run.status == msp.MSP_OK
    for i, inst in enumerate(insts):
        assert run.first_ms[i] >= 0.0
    # solutions found are exact
    res, sols, ctx = msp.solve(insts, mode=msp.MSP_FIRST, max_seconds=120.0)
    for i, inst in enumerate(insts):
        assert len(sols[i]) >= 1
        for x in sols[i].astype(np.int64):
            assert np.array_equal(x @ inst.A.T.astype(np.int64), inst.d)
    ctx.close()


def test_feature_log_is_finite_and_complete():
    insts = I.batch_m4_7(6)
    pk = I.pack(insts)
    msp = M()
    ctx = msp.Context(log_features=1)
    ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
    ctx.msp_reduce()
    ctx.msp_enumerate()
    for i in range(len(insts)):
        f = ctx.msp_export_features(i)
        p = ctx.msp_export_prefixes(i)
        assert f.shape == (len(p["u"]), 32)
        assert np.all(np.isfinite(f))
        assert np.all(f[:, 0] >= 0) and np.all(f[:, 0] <= 1.001)
    ctx.close()


def test_trained_scorer_gains_over_plain_order():
    """What the network buys: trained on m = 5..7 instances (seeds disjoint
    from the batch's), it ranks the subtrees of the batch's m = 6, 7
    instances so that the first subtree holding a solution moves far up the
    queue, and a walker taking the subtrees in that order spends fewer nodes
    before reaching it than in the depth-first order (geometric means over
    the instances; training is deterministic).  All-solutions results are
    unaffected (tested above)."""
    from paper_2508_08702_gb300 import learn
    data = learn.collect(I.training_set(256), split_target=2048)
    theta, losses = learn.train(data, steps=4000)
    held = [x for x in I.batch_m4_7(64) if x.m >= 6]
    w = learn.sequential_work_to_first(held, theta, split_target=2048)
    work, rank = w.ratios()
    print(f"learned / plain, geometric means over {len(held)} instances: work before the first "
          f"solution-bearing subtree {work:.3f}, its queue position {rank:.3f}")
    assert work < 0.8
    assert rank < 0.2
