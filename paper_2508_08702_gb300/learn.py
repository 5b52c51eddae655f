"""Training and use of the subtree scorer (the learned queue order).

The scorer only reorders the subtrees of the first-solution mode; it never
changes the pruning.  Data: the plain all-solutions enumeration logs, for
every subtree prefix, its 32 features and its outcome (did the subtree hold a
solution, how many nodes did it take).  Training: Adam on the device with the
library's own tensor-core forward/backward kernels (msp_mlp_train).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import instances as I
from . import msp as M

IN, HID, OUT = 32, 64, 8


@dataclass
class Dataset:
    x: np.ndarray        # (rows, 32) float32 features
    y: np.ndarray        # (rows, 2) float32: found (0/1), log(1 + nodes)
    instances: int

    @property
    def positives(self) -> int:
        return int(self.y[:, 0].sum())


def init_params(seed: int = 0) -> np.ndarray:
    """He initialisation; float32 vector W1[32][64] b1 W2[64][64] b2 W3[64][8] b3."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((IN, HID), (HID, HID), (HID, OUT)):
        parts.append(rng.normal(0.0, np.sqrt(2.0 / fan_in), size=(fan_in, fan_out)).reshape(-1))
        parts.append(np.zeros(fan_out))
    theta = np.concatenate(parts).astype(np.float32)
    assert theta.size == M.mlp_param_count()
    return theta


def collect(instances: Sequence, split_target: int = 16384, batch: int = 64, **opts) -> Dataset:
    """Plain all-solutions runs with feature logging; one row per prefix."""
    xs, ys = [], []
    for b0 in range(0, len(instances), batch):
        chunk = list(instances[b0:b0 + batch])
        pk = I.pack(chunk)
        ctx = M.Context(log_features=1, split_target=split_target, **opts)
        ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
        ctx.msp_reduce()
        ctx.msp_enumerate(M.MSP_ALL, M.MSP_PLAIN)
        for i in range(len(chunk)):
            f = ctx.msp_export_features(i)
            if len(f) == 0:
                continue
            p = ctx.msp_export_prefixes(i)
            xs.append(f)
            ys.append(np.stack([(p["sols"] > 0).astype(np.float32),
                                np.log1p(np.maximum(p["nodes"], 0)).astype(np.float32)], axis=1))
        ctx.close()
    return Dataset(np.concatenate(xs).astype(np.float32), np.concatenate(ys).astype(np.float32), len(instances))


def train(data: Dataset, steps: int = 4000, lr: float = 2e-3, seed: int = 0,
          pos_weight: Optional[float] = None) -> Tuple[np.ndarray, np.ndarray]:
    """Adam on the device; returns (theta, per-step mini-batch losses)."""
    import torch
    n = len(data.x)
    if pos_weight is None:   # balance the rare positive subtrees
        pos = max(1, data.positives)
        pos_weight = float(min(100.0, (n - pos) / pos))
    theta = torch.from_numpy(init_params(seed)).cuda()
    X = torch.from_numpy(np.ascontiguousarray(data.x)).cuda()
    Y = torch.from_numpy(np.ascontiguousarray(data.y)).cuda()
    losses = torch.zeros(steps, dtype=torch.float32, device="cuda")
    ctx = M.Context()
    ctx.msp_mlp_train(theta, X, Y, steps, lr, pos_weight, seed, losses)
    ctx.close()
    return theta.cpu().numpy(), losses.cpu().numpy()


@dataclass
class FirstRun:
    first_ms: List[float]     # per instance, -1 if not solved within the cap
    nodes: List[int]          # per instance, nodes evaluated until the run stopped
    total_ms: float
    status: int


def first_solution(instances: Sequence, order: int, scorer: Optional[np.ndarray] = None,
                   split_target: int = 0, time_cap_s: float = 0.0, **opts) -> FirstRun:
    """Time to the first verified solution of every instance of the batch
    (one launch; each instance stops on its own first solution)."""
    pk = I.pack(list(instances))
    ctx = M.Context(split_target=split_target, **opts)
    if scorer is not None:
        ctx.msp_set_scorer(scorer)
    ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
    ctx.msp_reduce()
    res = ctx.msp_enumerate(M.MSP_FIRST, order, time_cap_s, allow=(M.MSP_OK, M.MSP_ETIMEOUT))
    ph = ctx.msp_phase_ms()
    out = FirstRun([s["first_ms"] for s in res.stats], [s["nodes"] for s in res.stats],
                   ph["split"] + ph["enumerate"], res.status)
    ctx.close()
    return out


@dataclass
class OrderWork:
    plain: List[int]      # per instance: nodes of the subtrees taken before the first one holding a solution
    learned: List[int]
    plain_rank: List[int]     # per instance: queue position of the first subtree holding a solution
    learned_rank: List[int]
    prefixes: List[int]

    def ratios(self):
        """Geometric means over the instances with a solution of the learned
        / plain ratios of (work + 1) and of (rank + 1)."""
        p, l = np.array(self.plain, float), np.array(self.learned, float)
        pr, lr = np.array(self.plain_rank, float), np.array(self.learned_rank, float)
        ok = pr < np.array(self.prefixes)
        return (float(np.exp(np.mean(np.log((l[ok] + 1) / (p[ok] + 1))))),
                float(np.exp(np.mean(np.log((lr[ok] + 1) / (pr[ok] + 1))))))


def _work_before_first(nodes: np.ndarray, sols: np.ndarray, order: np.ndarray):
    hit = np.nonzero(sols[order] > 0)[0]
    stop = hit[0] if len(hit) else len(order)
    return int(nodes[order[:stop]].sum()), int(stop)


def sequential_work_to_first(instances: Sequence, scorer: np.ndarray, split_target: int = 0, **opts) -> OrderWork:
    """Deterministic measure of an order: the nodes a single walker taking
    the subtrees in that order spends before it reaches the first subtree
    that holds a solution.  Subtree sizes and outcomes come from one plain
    all-solutions run (logged per prefix); the learned order ranks the same
    prefixes by the scorer's priority, ties by depth-first position."""
    import torch
    pk = I.pack(list(instances))
    ctx = M.Context(log_features=1, split_target=split_target, **opts)
    ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
    ctx.msp_reduce()
    ctx.msp_enumerate(M.MSP_ALL, M.MSP_PLAIN)
    th = torch.from_numpy(np.ascontiguousarray(scorer, dtype=np.float32)).cuda()
    out = OrderWork([], [], [], [], [])
    for i in range(len(instances)):
        f = ctx.msp_export_features(i)
        p = ctx.msp_export_prefixes(i)
        k = len(f)
        out.prefixes.append(k)
        if k == 0:
            for a in (out.plain, out.learned, out.plain_rank, out.learned_rank):
                a.append(0)
            continue
        y = torch.zeros((k, OUT), dtype=torch.float32, device="cuda")
        ctx.msp_mlp_forward(th, torch.from_numpy(f).cuda(), y)
        pri = y.cpu().numpy()[:, 0]            # the queue priority (logit of P(solution))
        learned = np.lexsort((np.arange(k), -pri))
        w, r = _work_before_first(p["nodes"], p["sols"], np.arange(k))
        out.plain.append(w)
        out.plain_rank.append(r)
        w, r = _work_before_first(p["nodes"], p["sols"], learned)
        out.learned.append(w)
        out.learned_rank.append(r)
    ctx.close()
    return out
