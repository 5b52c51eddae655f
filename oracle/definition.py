"""The solution set by its plain definition (test infrastructure only).

fMSP (Sec. 1): the set {x in {0,1}^n : A x = d}.  Two exact ways to list it,
neither of which uses lattices:

* ``brute_force``  -- try all 2^n binary vectors (n <= 26);
* ``brute_force_bounds`` -- the general problem of Sec. 2 with bounds
  0 <= x_j <= r_j: try every point of the box (at most 2^22 points);
* ``meet_in_middle`` -- split the columns in two halves, list all 2^(n/2)
  partial sums of each half, and join the halves whose sums add up to d
  (Horowitz-Sahni style).  Exact: every candidate pair is verified on the
  full vector, so key collisions can only cost time (n <= 44).

Both return the solutions as a (count, n) uint8 array sorted
lexicographically, the same convention as the enumeration oracle.
"""
from __future__ import annotations

import numpy as np


def _sorted(x: np.ndarray, n: int) -> np.ndarray:
    if len(x) == 0:
        return np.zeros((0, n), np.uint8)
    keys = [x[:, c] for c in range(n - 1, -1, -1)]
    return x[np.lexsort(keys)].astype(np.uint8)


def _all_binary(k: int, start: int, stop: int) -> np.ndarray:
    idx = np.arange(start, stop, dtype=np.int64)
    return ((idx[:, None] >> np.arange(k, dtype=np.int64)) & 1).astype(np.int8)


def brute_force(A: np.ndarray, d: np.ndarray, chunk: int = 1 << 18) -> np.ndarray:
    A = np.asarray(A, dtype=np.int64)
    d = np.asarray(d, dtype=np.int64)
    m, n = A.shape
    if n > 26:
        raise ValueError("brute force is limited to n <= 26")
    found = []
    for start in range(0, 1 << n, chunk):
        X = _all_binary(n, start, min(1 << n, start + chunk))
        ok = np.all(X.astype(np.int64) @ A.T == d[None, :], axis=1)
        if ok.any():
            found.append(X[ok])
    x = np.concatenate(found) if found else np.zeros((0, n), np.int8)
    return _sorted(x, n)


def meet_in_middle(A: np.ndarray, d: np.ndarray, seed: int = 12345) -> np.ndarray:
    A = np.asarray(A, dtype=np.int64)
    d = np.asarray(d, dtype=np.int64)
    m, n = A.shape
    if n > 44:
        raise ValueError("meet in the middle is limited to n <= 44")
    h = n // 2
    k2 = n - h
    X1 = _all_binary(h, 0, 1 << h)
    X2 = _all_binary(k2, 0, 1 << k2)
    S1 = X1.astype(np.int64) @ A[:, :h].T            # (2^h, m)
    S2 = d[None, :] - X2.astype(np.int64) @ A[:, h:].T
    # random linear key; equal vectors always have equal keys
    rng = np.random.default_rng(seed)
    r = rng.integers(1, 1 << 20, size=m, dtype=np.int64)
    K1 = S1 @ r
    K2 = S2 @ r
    order = np.argsort(K1, kind="stable")
    K1s = K1[order]
    lo = np.searchsorted(K1s, K2, side="left")
    hi = np.searchsorted(K1s, K2, side="right")
    out = []
    for j in np.nonzero(hi > lo)[0]:
        for p in range(lo[j], hi[j]):
            i = order[p]
            if np.array_equal(S1[i], S2[j]):
                out.append(np.concatenate([X1[i], X2[j]]))
    x = np.array(out, dtype=np.int8).reshape(-1, n)
    return _sorted(x, n)


def solutions(A: np.ndarray, d: np.ndarray) -> np.ndarray:
    """The solution set by whichever exact method fits the size."""
    n = np.asarray(A).shape[1]
    return brute_force(A, d) if n <= 22 else meet_in_middle(A, d)


def brute_force_bounds(A: np.ndarray, d: np.ndarray, r: np.ndarray, chunk: int = 1 << 18) -> np.ndarray:
    """All integer x with A x = d and 0 <= x <= r (mixed-radix counting)."""
    A = np.asarray(A, dtype=np.int64)
    d = np.asarray(d, dtype=np.int64)
    r = np.asarray(r, dtype=np.int64)
    m, n = A.shape
    radix = r + 1
    total = int(np.prod(radix))
    if total > (1 << 22):
        raise ValueError("the box has more than 2^22 points")
    found = []
    for start in range(0, total, chunk):
        idx = np.arange(start, min(total, start + chunk), dtype=np.int64)
        X = np.zeros((len(idx), n), np.int64)
        rest = idx.copy()
        for c in range(n):
            X[:, c] = rest % radix[c]
            rest //= radix[c]
        ok = np.all(X @ A.T == d[None, :], axis=1)
        if ok.any():
            found.append(X[ok])
    x = np.concatenate(found) if found else np.zeros((0, n), np.int64)
    return _sorted(x, n)
