"""The element-wise gradient check of the GPU scorer tests, validated on the
CPU: it accepts a float32 computation with the scorer kernels' precision
contract (bfloat16 operands, float32 sums, the rounding points stated in
oracle/mlp.py) and rejects gradients with planted mistakes."""
import numpy as np
import pytest

from oracle import mlp as R
from tests.mlp_check import block_failures


def _f32_grad(theta, x, found, ln, pw, mistake=None):
    """The scorer's loss gradient evaluated in float32 with bfloat16 operands
    at the contract's rounding points; `mistake` plants one error."""
    f32 = np.float32
    b = lambda a: R.bf16(a).astype(f32)
    p = {k: v.astype(f32) for k, v in R.unpack(theta).items()}
    n = len(x)
    xb = b(x)
    a1 = (xb @ b(p["W1"])).astype(f32) + p["b1"]
    h1b = b(np.maximum(a1, 0))
    a2 = (h1b @ b(p["W2"])).astype(f32) + p["b2"]
    h2b = b(np.maximum(a2, 0))
    y = (h2b @ b(p["W3"])).astype(f32) + p["b3"]
    z = y[:, 0]
    w = np.where(found > 0.5, pw, 1.0).astype(f32)
    dy = np.zeros_like(y)
    dy[:, 0] = w * (f32(1) / (f32(1) + np.exp(-z)) - found) / f32(n)
    dy[:, 1] = f32(2 * R.NODE_WEIGHT) * (y[:, 1] - ln) / f32(n)
    if mistake == "swap_outputs":
        dy[:, [0, 1]] = dy[:, [1, 0]]
    dyb = b(dy)
    g = {"W3": h2b.T @ dyb, "b3": dy.sum(0)}
    m2 = (a2 > 0) if mistake != "no_mask2" else np.ones_like(a2, bool)
    W3b = b(p["W3"])
    dh2 = (dyb @ W3b.T) * m2
    g["W2"] = h1b.T @ b(dh2)
    g["b2"] = dh2.sum(0) * (-1 if mistake == "b2_sign" else 1)
    W2b = b(p["W2"])
    dh1 = (b(dh2) @ (W2b if mistake == "w2_not_transposed" else W2b.T)) * (a1 > 0)
    g["W1"] = xb.T @ b(dh1)
    g["b1"] = dh1.sum(0) * (n if mistake == "b1_no_mean" else 1)
    if mistake == "b3_zero":
        g["b3"] = np.zeros_like(g["b3"])
    return R.pack({k: np.asarray(v, np.float64) for k, v in g.items()})


def _case(n, seed):
    rng = np.random.default_rng(seed)
    theta = R.init(2) * 0.8
    theta[2048:2112] = rng.normal(0, 0.1, 64)
    x = rng.normal(0, 1, size=(n, 32)).astype(np.float32)
    found = (rng.random(n) < 0.2).astype(np.float32)
    ln = rng.normal(4, 1, n).astype(np.float32)
    return theta, x, found, ln


@pytest.mark.parametrize("n,seed", [(128, 1), (300, 2), (1037, 3)])
def test_check_accepts_float32_contract_arithmetic(n, seed):
    theta, x, found, ln = _case(n, seed)
    _, want, scale = R.loss_and_grad(theta, x, found, ln, 3.0, round_grad_bf16=True, scales=True)
    got = _f32_grad(theta, x, found, ln, 3.0)
    assert block_failures(got, want, scale, R.blocks) == []


@pytest.mark.parametrize("mistake,block", [("swap_outputs", "b3"), ("no_mask2", "b2"), ("b2_sign", "b2"),
                                           ("w2_not_transposed", "W1"), ("b1_no_mean", "b1"),
                                           ("b3_zero", "b3")])
def test_check_rejects_planted_mistakes(mistake, block):
    theta, x, found, ln = _case(300, 2)
    _, want, scale = R.loss_and_grad(theta, x, found, ln, 3.0, round_grad_bf16=True, scales=True)
    got = _f32_grad(theta, x, found, ln, 3.0, mistake=mistake)
    assert block in block_failures(got, want, scale, R.blocks)


def test_contract_rounding_stays_within_bf16_of_exact_backward():
    """The backward rounding points move each element by at most a few
    bfloat16 units of its scale against the unrounded backward (whose
    formulas are pinned by finite differences in test_oracle_mlp)."""
    theta, x, found, ln = _case(300, 4)
    _, g0, s0 = R.loss_and_grad(theta, x, found, ln, 3.0, scales=True)
    _, g1, s1 = R.loss_and_grad(theta, x, found, ln, 3.0, round_grad_bf16=True, scales=True)
    assert not np.array_equal(g0, g1)
    assert np.all(np.abs(g1 - g0) <= 3 * 2.0 ** -8 * np.maximum(s0, s1) + 1e-15)
