"""Host model of the fused launch's publication protocol (enum.cu,
publish_instance / find_entry): preparers reserve an entry and a range of
queue positions with one atomic, write the entry, then flag it ready;
walkers holding a queue position look for the entry whose range holds it,
reading only ready entries.  Checked over random interleavings, with
instances that publish no subtrees: a walker is never sent to a wrong
instance, and once every entry is ready every position below the total
resolves to its own instance."""
import random

import pytest


class Model:
    def __init__(self, sizes):
        self.count = len(sizes)
        self.sizes = sizes
        self.qres_count = 0
        self.qres_total = 0
        self.base = [None] * self.count      # rl[r]
        self.inst = [None] * self.count      # rl[count + r]
        self.ready = [0] * self.count        # rl[2 count + r]
        self.truth = {}                      # queue position -> instance

    # publish_instance, split into its visible steps
    def reserve(self, i):
        r, base = self.qres_count, self.qres_total
        self.qres_count += 1
        self.qres_total += self.sizes[i]
        for p in range(base, base + self.sizes[i]):
            self.truth[p] = i
        return r, base

    def write(self, r, i, base):
        self.base[r] = base
        self.inst[r] = i

    def flag(self, r):
        self.ready[r] = 1

    # find_entry on a snapshot of the reservation word
    def find(self, tk):
        r_res, reserved = self.qres_count, self.qres_total
        if tk >= reserved:
            return None
        if not self.ready[0]:
            return -1
        lo, hi = 0, r_res
        while hi - lo > 1:
            mid = (lo + hi) // 2
            if not self.ready[mid]:
                return -1
            if self.base[mid] <= tk:
                lo = mid
            else:
                hi = mid
        return self.inst[lo]


@pytest.mark.parametrize("seed", range(200))
def test_random_interleavings_never_misroute(seed):
    rng = random.Random(seed)
    count = rng.randint(1, 9)
    sizes = [rng.choice([0, 0, 1, 2, 5, 17]) for _ in range(count)]
    m = Model(sizes)
    # each preparer: reserve -> write -> flag, steps interleaved at random
    pending = {i: 0 for i in range(count)}
    state = {}
    total = sum(sizes)
    while pending:
        i = rng.choice(list(pending))
        step = pending[i]
        if step == 0:
            state[i] = m.reserve(i)
        elif step == 1:
            m.write(state[i][0], i, state[i][1])
        else:
            m.flag(state[i][0])
        pending[i] += 1
        if pending[i] == 3:
            del pending[i]
        # walkers probe arbitrary positions at every point of the interleaving
        for tk in range(total + 2):
            got = m.find(tk)
            if got is not None and got != -1:
                assert got == m.truth[tk], (seed, tk, got)
    for tk in range(total):
        assert m.find(tk) == m.truth[tk]
    assert m.find(total) is None
