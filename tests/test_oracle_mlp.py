"""Pins for the scorer's CPU reference (oracle/mlp.py).

The loss gradient is checked against central finite differences of the
loss on the exact (unrounded) network -- a wrong sign, a dropped term or a
transposed weight in the backward formulas fails here -- and the bfloat16
rounding against values worked out by hand."""
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
    idx = rng.choice(R.MLP_PARAMS, size=80, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fp, _ = R.loss_and_grad(tp, x, found, ln, pos_weight, round_bf16=False)
        fm, _ = R.loss_and_grad(tm, x, found, ln, pos_weight, round_bf16=False)
        num = (fp - fm) / (2 * h)
        assert num == pytest.approx(g[i], rel=1e-5, abs=1e-8), i


def test_score_ranks_by_solution_probability():
    y = np.zeros((3, 8))
    y[:, 0] = [2.0, 2.5, -2.0]
    y[:, 1] = [1.0, 5.0, 1.0]
    s = R.score(y)
    assert s[1] > s[0] > s[2]
