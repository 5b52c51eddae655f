"""Pins for the scorer's CPU reference (oracle/mlp.py).

The loss gradient is checked against central finite differences of the
loss on the exact (unrounded) network -- a wrong sign, a dropped term or a
transposed weight in the backward formulas fails here -- and the forward
pass and the bfloat16 rounding against values worked out by hand."""
import math

import numpy as np
import pytest

from oracle import mlp as R


def test_bf16_rounding_by_hand():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5, 1.0 + 2.0 ** -7 + 2.0 ** -8, 0.0])
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7 -> even mantissa (1); 1 + 3*2^-9
    # rounds up to 1 + 2^-7; 1 + 2^-7 + 2^-8 is a tie -> even (1 + 2^-6)
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -7, -2.5, 1.0 + 2.0 ** -6, 0.0])
    assert np.array_equal(R.bf16(x), want)


def test_param_count_and_layout():
    assert R.MLP_PARAMS == 32 * 64 + 64 + 64 * 64 + 64 + 64 * 8 + 8 == 6792
    th = np.arange(R.MLP_PARAMS, dtype=np.float64)
    p = R.unpack(th)
    assert p["W1"][0, 1] == 1 and p["b1"][0] == 2048 and p["W2"][0, 0] == 2112 and p["b3"][7] == 6791
    assert np.array_equal(R.pack(p), th)


@pytest.mark.parametrize("pos_weight", [1.0, 7.5])
def test_gradient_matches_finite_differences(pos_weight):
    rng = np.random.default_rng(3)
    theta = R.init(5).astype(np.float64) * 0.7
    theta[2048:2112] = rng.normal(0, 0.1, 64)
    x = rng.normal(0, 1, size=(9, 32))
    found = (rng.random(9) < 0.4).astype(np.float64)
    ln = rng.normal(3, 1, 9)
    _, g = R.loss_and_grad(theta, x, found, ln, pos_weight, round_bf16=False)
    # 12 indices from every parameter block (all of b3): a uniform sample
    # of 80 out of 6792 would leave the 64-entry biases mostly unchecked
    idx, o = [], 0
    for _, shape in R.SHAPES:
        size = int(np.prod(shape))
        idx.extend((o + rng.choice(size, size=min(12, size), replace=False)).tolist())
        o += size
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fp, _ = R.loss_and_grad(tp, x, found, ln, pos_weight, round_bf16=False)
        fm, _ = R.loss_and_grad(tm, x, found, ln, pos_weight, round_bf16=False)
        num = (fp - fm) / (2 * h)
        assert num == pytest.approx(g[i], rel=1e-5, abs=1e-8), i


@pytest.mark.parametrize("round_bf16", [False, True])
def test_forward_by_hand(round_bf16):
    """A network with a handful of nonzero weights, every value exact in
    bfloat16, worked out by hand (32 -> 64 -> 64 -> 8, ReLU, row = input):
      layer 1: a = (2 * 1.5 + 0.5, -1 * 3 + 0.25) = (3.5, -2.75) -> h1 = (3.5, 0)
      layer 2: a = (1 * 3.5, -2 * 3.5 + 1, 0.75, -1 * 0) = (3.5, -6, 0.75, 0)
               -> h2 = (3.5, 0, 0.75, 0)
      layer 3: y0 = 2 * 3.5 - 1 = 6, y1 = 4 * 0.75 + 0.5 = 3.5, y2 = 8 * 0 = 0,
               y3 = 1 * 0 = 0, y7 = b3[7] = -0.125
    A missing ReLU (y2 = -48 or y3 = 2.75), a transposed layer or a dropped
    bias changes y."""
    theta, x = _hand_network()
    y, _ = R.forward(theta, x, round_bf16=round_bf16)
    want = np.zeros((2, 8))
    want[0, :3] = [6.0, 3.5, 0.0]
    want[:, 7] = -0.125
    # the second row's input is zero: h1 = relu(b1) = (0.5, 0.25),
    # h2 = relu(0.5, -2 * 0.5 + 1, 0.75, -0.25) = (0.5, 0, 0.75, 0)
    h1 = np.array([0.5, 0.25])
    h2 = np.array([h1[0], -2 * h1[0] + 1.0, 0.75])
    want[1, 0] = 2 * h2[0] - 1.0
    want[1, 1] = 4 * h2[2] + 0.5
    want[1, 2] = 8 * max(h2[1], 0.0)
    assert np.array_equal(y, want)


def _hand_network():
    """The network of test_forward_by_hand."""
    p = R.unpack(np.zeros(R.MLP_PARAMS))
    p["W1"][0, 0], p["W1"][1, 1] = 2.0, -1.0
    p["b1"][0], p["b1"][1] = 0.5, 0.25
    p["W2"][0, 0], p["W2"][0, 1], p["W2"][1, 3] = 1.0, -2.0, -1.0
    p["b2"][1], p["b2"][2] = 1.0, 0.75
    p["W3"][0, 0], p["W3"][2, 1], p["W3"][1, 2], p["W3"][3, 3] = 2.0, 4.0, 8.0, 1.0
    p["b3"][0], p["b3"][1], p["b3"][7] = -1.0, 0.5, -0.125
    x = np.zeros((2, 32))
    x[0, 0], x[0, 1] = 1.5, 3.0
    return R.pack(p), x


def test_loss_by_hand():
    """The loss of the documented contract on the network above (outputs
    y = (6, 3.5) and (0, 3.5)): per row pos_weight * BCE(y0, found) for
    found rows, BCE otherwise, plus 0.1 (y1 - log(1 + nodes))^2, averaged.
      row 0: found, pos_weight 2: 2 log(1 + e^-6) + 0.1 (3.5 - 3.5)^2
      row 1: not found:           log 2           + 0.1 (3.5 - 1.5)^2 = log 2 + 0.4"""
    theta, x = _hand_network()
    loss, _ = R.loss_and_grad(theta, x, np.array([1.0, 0.0]), np.array([3.5, 1.5]), pos_weight=2.0)
    want = (2 * math.log1p(math.exp(-6.0)) + math.log(2.0) + 0.4) / 2
    assert loss == pytest.approx(want, rel=1e-12)


def test_score_ranks_by_solution_probability():
    y = np.zeros((3, 8))
    y[:, 0] = [2.0, 2.5, -2.0]
    y[:, 1] = [1.0, 5.0, 1.0]
    s = R.score(y)
    assert s[1] > s[0] > s[2]
