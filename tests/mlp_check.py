"""Element-wise comparison of scorer gradients, block by block.

A gradient element of the scorer is a sum over the mini-batch rows of
products a_r g_r (a weight) or of terms g_r (a bias).  Computed in float32
from bfloat16 operands it differs from the float64 value of the same
bfloat16 operands by the float32 accumulation error, at most about
rows x 2^-24 x S, where S = sum_r |a_r g_r| (resp. sum_r |g_r|) is the
element's scale.  Rarely an operand computed in float32 lands on the other
side of a bfloat16 rounding boundary than its float64 value: it then moves by
one bfloat16 unit (2^-8 of its size) and shifts the elements it feeds by at
most a few 2^-8 S.  Hence the check, per parameter block:
  * at least `frac` of the elements within 2^-14 S (float32-level agreement),
  * every element within 2^-5 S,
each with an absolute floor of 2^-20 x the block's largest scale.  A wrong
formula (a dropped mask, a transposed weight, a wrong sign, a missing 1/B)
moves elements by a large part of S and fails the second test.
"""
from __future__ import annotations

import numpy as np

TIGHT = 2.0 ** -14
LOOSE = 2.0 ** -5
FRAC = 0.97


def block_failures(got: np.ndarray, want: np.ndarray, scale: np.ndarray, blocks) -> list:
    """Names of the blocks that fail the check (empty: all pass).  `blocks`
    maps a flat vector to {name: block} (oracle.mlp.blocks)."""
    G, W, S = blocks(got), blocks(want), blocks(scale)
    bad = []
    for name in W:
        err = np.abs(G[name] - W[name])
        floor = 2.0 ** -20 * max(float(S[name].max()), 1e-30)
        tight = err <= TIGHT * S[name] + floor
        loose = err <= LOOSE * S[name] + floor
        if tight.mean() < FRAC or not loose.all():
            bad.append(name)
    return bad
