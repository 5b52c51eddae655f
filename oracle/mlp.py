"""Plain numpy reference of the subtree scorer (test infrastructure only).

The scorer is not part of the paper: it only reorders the queue of subtrees
(prefixes) for the first-solution mode and never changes the pruning.  This
module is the CPU definition the CUDA kernels are checked against.

Network: x (32 features) -> relu(x W1 + b1) (64) -> relu(h1 W2 + b2) (64)
-> y = h2 W3 + b3 (8 outputs, 2 used: y0 = logit of P(the subtree holds a
solution), y1 = predicted log(1 + nodes of the subtree)).

Precision contract (the kernels' tensor-core path): every product takes
bfloat16 operands and accumulates in float32.  Forward: inputs, weights and
the hidden activations fed to the next layer are rounded to bfloat16 (round
to nearest even).  Backward (``round_grad_bf16=True``): the back-propagated
signals dL/dy, dL/da2 and dL/da1 are rounded to bfloat16 where they enter a
product (the next backward product and the weight-gradient products), while
the bias gradients sum the unrounded signals.  Sums, biases, activations
before rounding and all gradients are exact here (float64) where the kernels
use float32.

Loss per row: pos_weight * BCE(y0, found) for found rows, BCE for the
others, plus 0.1 * (y1 - log1p(nodes))^2; the batch loss is the mean.

Parameter vector layout (float32, MLP_PARAMS entries):
W1[32][64], b1[64], W2[64][64], b2[64], W3[64][8], b3[8]   (row = input).
"""
from __future__ import annotations

import numpy as np

IN, HID, OUT = 32, 64, 8
SHAPES = [("W1", (IN, HID)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (HID, OUT)), ("b3", (OUT,))]
MLP_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
NODE_WEIGHT = 0.1


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def bf16(a: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def init(seed: int = 0) -> np.ndarray:
    """He-style initialisation (float32 master parameters)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SHAPES:
        if name.startswith("W"):
            p[name] = rng.normal(0.0, np.sqrt(2.0 / shape[0]), size=shape)
        else:
            p[name] = np.zeros(shape)
    return pack(p).astype(np.float32)


def forward(theta: np.ndarray, x: np.ndarray, round_bf16: bool = True):
    """round_bf16=False gives the exact (unrounded) network, used to pin the
    derivative formulas against finite differences."""
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    p = unpack(theta)
    xb = r(x)
    a1 = xb @ r(p["W1"]) + p["b1"]
    h1 = np.maximum(a1, 0.0)
    h1b = r(h1)
    a2 = h1b @ r(p["W2"]) + p["b2"]
    h2 = np.maximum(a2, 0.0)
    h2b = r(h2)
    y = h2b @ r(p["W3"]) + p["b3"]
    return y, dict(xb=xb, a1=a1, h1b=h1b, a2=a2, h2b=h2b)


def loss_and_grad(theta: np.ndarray, x: np.ndarray, found: np.ndarray, lognodes: np.ndarray,
                  pos_weight: float = 1.0, round_bf16: bool = True, round_grad_bf16: bool = False,
                  scales: bool = False):
    """Mean loss over the rows and its gradient with respect to theta (the
    derivative is taken through the rounded values as constants, as the
    kernels do).  round_grad_bf16: also round the back-propagated signals to
    bfloat16 where they enter a product (the backward half of the precision
    contract).  scales: also return, per parameter, the sum over the rows of
    the absolute values of the terms that make up its gradient (|A|^T |G|
    for a weight, sum |G| for a bias) -- the size against which rounding
    errors of that element are measured."""
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    rg = bf16 if round_grad_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    p = unpack(theta)
    y, c = forward(theta, x, round_bf16)
    B = x.shape[0]
    z, f = y[:, 0], found.astype(np.float64)
    w = np.where(f > 0.5, pos_weight, 1.0)
    # BCE with logits, stable form
    bce = np.maximum(z, 0) - z * f + np.log1p(np.exp(-np.abs(z)))
    diff = y[:, 1] - lognodes
    loss = float(np.mean(w * bce + NODE_WEIGHT * diff * diff))
    dy = np.zeros_like(y)
    dy[:, 0] = w * (1.0 / (1.0 + np.exp(-z)) - f) / B
    dy[:, 1] = 2.0 * NODE_WEIGHT * diff / B
    g, sc = {}, {}
    dyr = rg(dy)
    g["W3"] = c["h2b"].T @ dyr
    g["b3"] = dy.sum(axis=0)
    dh2 = (dyr @ r(p["W3"]).T) * (c["a2"] > 0)
    dh2r = rg(dh2)
    g["W2"] = c["h1b"].T @ dh2r
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2r @ r(p["W2"]).T) * (c["a1"] > 0)
    dh1r = rg(dh1)
    g["W1"] = c["xb"].T @ dh1r
    g["b1"] = dh1.sum(axis=0)
    if not scales:
        return loss, pack(g)
    sc["W3"] = np.abs(c["h2b"]).T @ np.abs(dyr)
    sc["b3"] = np.abs(dy).sum(axis=0)
    sc["W2"] = np.abs(c["h1b"]).T @ np.abs(dh2r)
    sc["b2"] = np.abs(dh2).sum(axis=0)
    sc["W1"] = np.abs(c["xb"]).T @ np.abs(dh1r)
    sc["b1"] = np.abs(dh1).sum(axis=0)
    return loss, pack(g), pack(sc)


def blocks(theta: np.ndarray) -> dict:
    """The parameter vector split into its named blocks (flat float64 views)."""
    return {name: v.reshape(-1) for name, v in unpack(theta).items()}


def score(y: np.ndarray) -> np.ndarray:
    """Queue priority: the logit of P(the subtree holds a solution).  The
    node-count output is an auxiliary training target only: ranking by P
    discounted by the predicted size reached the solution-bearing subtree
    later than ranking by P alone on held-out instances."""
    return y[:, 0]
