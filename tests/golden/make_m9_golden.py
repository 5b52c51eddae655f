"""Write the expected all-solutions results of the m = 9, n = 80, D = 100
workload (8 instances, seeds 4000..4007, planted x with exactly 40 ones) to
``m9_n80_d100_bkz10.txt`` beside this script.

Only the CPU oracle is called: the lattice of Eq. (2), LLL, extraction and
Gram-Schmidt (Alg. 1 steps 1-3), BKZ-10 of the kernel basis (Sec. 2), then
Algorithm 1 over the whole tree with the |w|_1 summation order of 16-lane
walkers (the width the GPU picks for n + 1 > 64).  Every solution must
satisfy A x = d (the fMSP definition of Sec. 1), which is checked before
anything is written.  One instance takes about an hour of one CPU core, so
the instances run in a process pool, one per core.

    python tests/golden/make_m9_golden.py [--jobs N]
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from tests.golden.m9_golden import PATH as OUT, basis_digest  # noqa: E402
LANES = 16
BETA = 10




def _job(i: int):
    from oracle import oracle as O
    from paper_2508_08702_gb300 import instances as I
    inst = I.m9_n80(8)[i]
    t0 = time.time()
    _, kern, _ = O.reduce(inst.A, inst.d)
    kb = O.bkz(kern, BETA).kern
    r = O.enumerate(kb, O.gso(kb), inst.A, inst.d, lanes=LANES, sol_cap=1 << 20)
    A = inst.A.astype(np.int64)
    for x in r.solutions.astype(np.int64):
        assert set(np.unique(x)) <= {0, 1} and np.array_equal(A @ x, inst.d), "oracle solution fails A x = d"
    assert any(np.array_equal(inst.planted, x) for x in r.solutions), "planted x missing"
    return dict(seed=inst.seed, nodes=r.nodes, passed=r.passed, leaves=r.leaves,
                sols=["".join(str(int(v)) for v in x) for x in r.solutions],
                digest=basis_digest(kb), seconds=time.time() - t0)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=min(8, os.cpu_count() or 1))
    args = ap.parse_args()
    with mp.get_context("spawn").Pool(args.jobs) as pool:
        res = pool.map(_job, range(8), chunksize=1)
    lines = [
        "# All binary solutions of A x = d (Sec. 1, fMSP) for the m = 9, n = 80, D = 100 workload:",
        "# seeds 4000..4007, A uniform in [0, 100), a planted x with exactly 40 ones, d = A x.",
        "# Written by tests/golden/make_m9_golden.py, which calls only the CPU oracle:",
        "# Eq. (2) lattice, LLL (delta 0.99), extraction, BKZ-10 of the kernel basis (Sec. 2),",
        f"# Gram-Schmidt (Eq. (4)), Algorithm 1 over the whole tree, |w|_1 order of {LANES}-lane walkers.",
        "# inst <seed> nodes <evaluated nodes> passed <norm-test passes> leaves <leaves> nsol <count> basis_sha256 <digest>",
        "# sol <seed> <x_1 ... x_n as 0/1 characters>   (lexicographic order)",
    ]
    for r in res:
        lines.append(f"inst {r['seed']} nodes {r['nodes']} passed {r['passed']} leaves {r['leaves']} "
                     f"nsol {len(r['sols'])} basis_sha256 {r['digest']}")
        lines += [f"sol {r['seed']} {s}" for s in r["sols"]]
        print(f"seed {r['seed']}: {r['nodes']} nodes, {len(r['sols'])} solutions, {r['seconds']:.0f} s", flush=True)
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
