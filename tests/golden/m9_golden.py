"""Reader of m9_n80_d100_bkz10.txt, the stored oracle results of the m = 9,
n = 80, D = 100 workload (see make_m9_golden.py, which writes it)."""
from __future__ import annotations

import hashlib
import os
from dataclasses import dataclass, field
from typing import Dict

import numpy as np

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "m9_n80_d100_bkz10.txt")


def basis_digest(kb: np.ndarray) -> str:
    """sha256 of a reduced kernel basis as little-endian int32, row-major."""
    return hashlib.sha256(np.ascontiguousarray(kb, dtype="<i4").tobytes()).hexdigest()


@dataclass
class Stored:
    nodes: int
    passed: int
    leaves: int
    digest: str
    solutions: np.ndarray          # (count, n) uint8, lexicographic order


@dataclass
class Golden:
    lanes: int
    instances: Dict[int, Stored] = field(default_factory=dict)


def load(path: str = PATH) -> Golden:
    lanes = None
    rows: Dict[int, dict] = {}
    with open(path) as f:
        for line in f:
            w = line.split()
            if not w:
                continue
            if w[0] == "#":
                if "-lane walkers" in line:
                    lanes = int(line.split("-lane walkers")[0].split()[-1])
                continue
            if w[0] == "inst":
                kv = dict(zip(w[2::2], w[3::2]))
                rows[int(w[1])] = dict(nodes=int(kv["nodes"]), passed=int(kv["passed"]), leaves=int(kv["leaves"]),
                                       nsol=int(kv["nsol"]), digest=kv["basis_sha256"], sols=[])
            elif w[0] == "sol":
                rows[int(w[1])]["sols"].append(np.frombuffer(w[2].encode(), np.uint8) - ord("0"))
    g = Golden(lanes=lanes)
    for seed, r in rows.items():
        assert len(r["sols"]) == r["nsol"], seed
        sols = np.array(r["sols"], dtype=np.uint8).reshape(len(r["sols"]), -1)
        g.instances[seed] = Stored(r["nodes"], r["passed"], r["leaves"], r["digest"], sols)
    return g
