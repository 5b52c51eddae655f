"""Seeded synthetic market-split instances.

This module is the one piece shared by the CUDA path, the CPU oracle and the
benchmark.  It only draws random numbers and packs them; it holds none of the
method's arithmetic (no lattice, no reduction, no enumeration).

Instances follow the shape of the QOBLIB market-split classes described in
Sec. 1 of the paper: n = 10(m-1) columns, entries a_ij uniform in [0, D),
D in {50, 100, 200}.  QOBLIB guarantees feasibility without saying how
(Sec. 1); here every instance is made feasible by planting a binary x and
setting d = A x.  The QOBLIB files themselves are not available, so these
seeded instances stand in for them.

Every generator uses ``numpy.random.default_rng(seed)`` (PCG64), so the
same seed gives the same instance on every machine.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Instance:
    """One fMSP instance A x = d, x in {0,1}^n (Sec. 1, feasibility form)."""

    A: np.ndarray            # int32, shape (m, n), row-major
    d: np.ndarray            # int64, shape (m,)
    planted: Optional[np.ndarray]   # uint8, shape (n,), one known solution (None: none planted)
    seed: int
    D: int
    tag: str = ""
    r: Optional[np.ndarray] = None   # int32 (n,) upper bounds 0 <= x <= r; None: binary

    @property
    def m(self) -> int:
        return int(self.A.shape[0])

    @property
    def n(self) -> int:
        return int(self.A.shape[1])


def _planted(rng: np.random.Generator, n: int, ones: Optional[int]) -> np.ndarray:
    if ones is None:
        return rng.integers(0, 2, size=n).astype(np.uint8)
    x = np.zeros(n, dtype=np.uint8)
    x[rng.permutation(n)[:ones]] = 1
    return x


def make_instance(seed: int, m: int, n: int, D: int, ones: Optional[int] = None,
                  tag: str = "") -> Instance:
    """A uniform in [0, D), a planted binary x (Bernoulli(1/2), or exactly
    ``ones`` ones at random positions), and d = A x."""
    rng = np.random.default_rng(seed)
    A = rng.integers(0, D, size=(m, n)).astype(np.int32)
    x = _planted(rng, n, ones)
    d = (A.astype(np.int64) @ x.astype(np.int64)).astype(np.int64)
    return Instance(A=A, d=d, planted=x, seed=seed, D=D, tag=tag)


# --- the five workloads -----------------------------------------------------

def single_m3() -> List[Instance]:
    """One instance m=3, n=20, D=100 (seed 1001)."""
    return [make_instance(1001, 3, 20, 100, tag="m3n20")]


def batch_m4_7(count: int = 64, first_seed: int = 2000) -> List[Instance]:
    """``count`` instances, m drawn uniformly from {4,5,6,7} by each seed's
    generator, n = 10(m-1), D cycling over {50, 100, 200}."""
    out = []
    for i in range(count):
        seed = first_seed + i
        rng = np.random.default_rng(seed)
        m = int(rng.integers(4, 8))
        n = 10 * (m - 1)
        D = (50, 100, 200)[i % 3]
        A = rng.integers(0, D, size=(m, n)).astype(np.int32)
        x = rng.integers(0, 2, size=n).astype(np.uint8)
        d = (A.astype(np.int64) @ x.astype(np.int64)).astype(np.int64)
        out.append(Instance(A=A, d=d, planted=x, seed=seed, D=D, tag=f"batch{i}"))
    return out


def m8_n70(count: int = 16) -> List[Instance]:
    """m=8, n=70, D=200, seeds 3000.. (planted Bernoulli(1/2))."""
    return [make_instance(3000 + i, 8, 70, 200, tag=f"m8n70_{i}") for i in range(count)]


def m9_n80(count: int = 8) -> List[Instance]:
    """m=9, n=80, D=100, seeds 4000..; the planted x has exactly 40 ones."""
    return [make_instance(4000 + i, 9, 80, 100, ones=40, tag=f"m9n80_{i}") for i in range(count)]


def m12_n110(count: int = 4) -> List[Instance]:
    """m=12, n=110, D=100, seeds 5000.. (planted Bernoulli(1/2))."""
    return [make_instance(5000 + i, 12, 110, 100, tag=f"m12n110_{i}") for i in range(count)]


def m12_n110_d50(count: int = 4) -> List[Instance]:
    """m=12, n=110, D=50, seeds 5100.. (planted Bernoulli(1/2)): the shape of
    the paper's only m = 12 row (D = 50)."""
    return [make_instance(5100 + i, 12, 110, 50, tag=f"m12d50_{i}") for i in range(count)]


def m10_n90_d50(count: int = 4) -> List[Instance]:
    """m=10, n=90, D=50, seeds 5200.. (planted Bernoulli(1/2)): the shape of
    the paper's (10, 90, 50) row."""
    return [make_instance(5200 + i, 10, 90, 50, tag=f"m10d50_{i}") for i in range(count)]


def m11_n100_d50(count: int = 4) -> List[Instance]:
    """m=11, n=100, D=50, seeds 5300.. (planted Bernoulli(1/2)): the shape of
    the paper's (11, 100, 50) row."""
    return [make_instance(5300 + i, 11, 100, 50, tag=f"m11d50_{i}") for i in range(count)]


def training_set(count: int = 256, first_seed: int = 30000) -> List[Instance]:
    """Training instances for the subtree scorer: m cycling 5,6,7, D cycling
    over {50, 100, 200}; seeds disjoint from every evaluation set."""
    out = []
    for i in range(count):
        m = 5 + (i % 3)
        D = (50, 100, 200)[(i // 3) % 3]
        out.append(make_instance(first_seed + i, m, 10 * (m - 1), D, tag=f"train{i}"))
    return out


def small(seed: int, m: int, n: int, D: int) -> Instance:
    """Small instances for brute-force checks (n <= 24)."""
    return make_instance(seed, m, n, D, tag=f"small_m{m}n{n}D{D}")


def bounded(seed: int, m: int, n: int, D: int, bounds=(1, 2, 3)) -> Instance:
    """The general problem of Sec. 2: 0 <= x_j <= r_j with r_j drawn from
    ``bounds``, A uniform in [0, D), a planted x uniform in the box, d = A x."""
    rng = np.random.default_rng(seed)
    A = rng.integers(0, D, size=(m, n)).astype(np.int32)
    r = rng.choice(np.asarray(bounds, dtype=np.int32), size=n).astype(np.int32)
    x = np.array([rng.integers(0, int(rj) + 1) for rj in r], dtype=np.uint8)
    d = (A.astype(np.int64) @ x.astype(np.int64)).astype(np.int64)
    return Instance(A=A, d=d, planted=x, seed=seed, D=D, tag=f"bounded_m{m}n{n}D{D}_{seed}", r=r)


def cornuejols_dawande(seed: int, m: int, D: int = 100) -> Instance:
    """The original market split instances (Sec. 1): n = 10(m-1), a_ij
    uniform in [0, D) (D = 100 in the original), d_i = floor(sum_j a_ij / 2).
    Nothing is planted, so feasibility is not known in advance: at m = 3..6
    about a third of them have no solution, and answering those takes an
    exhaustive search."""
    rng = np.random.default_rng(seed)
    n = 10 * (m - 1)
    A = rng.integers(0, D, size=(m, n)).astype(np.int32)
    d = (A.astype(np.int64).sum(axis=1) // 2).astype(np.int64)
    return Instance(A=A, d=d, planted=None, seed=seed, D=D, tag=f"cd_m{m}_D{D}_{seed}")


def centred(m: int, D: int = 50, count: int = 4, first_seed: int = 60000) -> List[Instance]:
    """Stand-ins for the paper's instance library at the rows of its timing
    table (Sec. 4): a_ij uniform in [0, D), n = 10(m-1) and the centred
    right-hand side d_i = floor(sum_j a_ij / 2) of the original construction;
    seeds first_seed + 100 m + D + i.  Their solution counts match the
    paper's table where it lists them (m = 7..9: e.g. 170-270 solutions per
    instance at m = 7, D = 50 and 670-860 at m = 8, D = 50, against the
    table's 25-306 and 752-1265), while instances with a planted Bernoulli(1/2)
    x have a tenth as many (7-66 and 10-199): their d lies off the centre of
    the distribution of A x.  Feasibility is not guaranteed by construction;
    a found solution proves it."""
    return [cornuejols_dawande(first_seed + 100 * m + D + i, m, D) for i in range(count)]


def cd_batch(m: int, count: int, first_seed: int = 9000) -> List[Instance]:
    """Cornuejols-Dawande instances of one m, seeds first_seed + m * 100 + i."""
    return [cornuejols_dawande(first_seed + m * 100 + i, m) for i in range(count)]


# --- packing for the batched C-ABI -------------------------------------------

@dataclass
class Packed:
    """Concatenated instances: dims[i] = (m_i, n_i); A and d back to back."""

    dims: np.ndarray                 # int32 (count, 2)
    A: np.ndarray                    # int32 (sum m_i n_i,)
    d: np.ndarray                    # int64 (sum m_i,)
    instances: List[Instance] = field(default_factory=list)
    r: Optional[np.ndarray] = None   # int32 (sum n_i,) upper bounds, None when all binary


def pack(instances: List[Instance]) -> Packed:
    dims = np.array([[x.m, x.n] for x in instances], dtype=np.int32).reshape(-1, 2)
    A = np.concatenate([x.A.reshape(-1) for x in instances]).astype(np.int32) if instances \
        else np.zeros(0, np.int32)
    d = np.concatenate([x.d.reshape(-1) for x in instances]).astype(np.int64) if instances \
        else np.zeros(0, np.int64)
    r = None
    bounds = [getattr(x, "r", None) for x in instances]
    if any(b is not None for b in bounds):
        r = np.concatenate([b if b is not None else np.ones(x.n, np.int32)
                            for b, x in zip(bounds, instances)]).astype(np.int32)
        r = np.ascontiguousarray(r)
    return Packed(dims=np.ascontiguousarray(dims), A=np.ascontiguousarray(A),
                  d=np.ascontiguousarray(d), instances=list(instances), r=r)
