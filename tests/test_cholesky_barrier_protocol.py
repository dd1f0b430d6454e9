"""The named-barrier protocol of the pipelined Cholesky in csrc/krp_gram.cu (chol_pipelined),
restated on the host and run under random warp schedules for every R up to 32.

Warp 0 posts "row j of U, V written" (bar.arrive) on barrier 1 (j even) or 3 (j odd) and waits
for "step s applied to rows >= s + 2" (bar.sync) on barrier 2 (s even) or 4 (s odd); warps 1-7
do the converse.  A hardware barrier of 256 threads completes a generation once 8 warps have
arrived, whichever generation each warp meant, so the protocol is correct only if no
generation ever collects arrivals meant for two different events, and no warp waits forever.
The test also checks that the single-barrier version of the same protocol fails that check."""
import random

import pytest


def _programs(R, alternate=True):
    row_bar = (lambda j: 1 + 2 * (j & 1)) if alternate else (lambda j: 1)
    step_bar = (lambda s: 2 + 2 * (s & 1)) if alternate else (lambda s: 2)
    progs = {0: [("arrive", row_bar(0), ("row", 0))]}
    for j in range(1, R):
        if j >= 2:
            progs[0].append(("sync", step_bar(j - 2), ("step", j - 2)))
        progs[0].append(("arrive", row_bar(j), ("row", j)))
    for w in range(1, 8):
        p = []
        for s in range(R - 1):
            p.append(("sync", row_bar(s), ("row", s)))
            if s + 2 < R:
                p.append(("arrive", step_bar(s), ("step", s)))
        p.append(("sync", row_bar(R - 1), ("row", R - 1)))
        progs[w] = p
    return progs


def _run(R, seed, alternate=True):
    """Executes the programs under a random interleaving; raises on a mixed generation or a
    deadlock."""
    rng = random.Random(seed)
    progs = _programs(R, alternate)
    pc = {w: 0 for w in progs}
    waiting = {}
    pending = {}
    while True:
        ready = [w for w in progs if pc[w] < len(progs[w]) and w not in waiting]
        if not ready:
            if waiting:
                raise RuntimeError(f"deadlock at R={R}")
            return
        w = rng.choice(ready)
        op, bar, tag = progs[w][pc[w]]
        pc[w] += 1
        pending.setdefault(bar, []).append((w, tag))
        if op == "sync":
            waiting[w] = bar
        if len(pending[bar]) == 8:  # 256 threads: the generation completes
            tags = {t for _, t in pending[bar]}
            if len(tags) != 1:
                raise AssertionError(f"barrier {bar} mixed {sorted(tags)} at R={R}")
            for ww, _ in pending[bar]:
                if waiting.get(ww) == bar:
                    del waiting[ww]
            pending[bar] = []


@pytest.mark.parametrize("R", list(range(1, 33)))
def test_alternating_barriers_never_mix_generations(R):
    for seed in range(60):
        _run(R, seed)


def test_single_barrier_per_role_would_mix_generations():
    with pytest.raises(AssertionError):
        for seed in range(200):
            _run(8, seed, alternate=False)
