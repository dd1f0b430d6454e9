"""Pins of the oracle's TTM schedules against the paper's flop tables
(Tables 1-6, Corollary 1) and against brute-force leaves."""
import json
import os

import numpy as np
import pytest

from oracle import cpqr_oracle as o

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ttm_flop_tables.json")))
TREES = {"none": o.TREE_NONE, "standard": o.TREE_STANDARD, "restructured": o.TREE_RESTRUCTURED}


def _poly(counts):
    return {(tuple(F), p): 2 * c for (F, p), c in counts.items()}


@pytest.mark.parametrize("case", GOLD["cases"], ids=lambda c: f"N{c['N']}-{c['tree']}")
def test_three_sweep_flop_polynomial_matches_paper(case):
    N = case["N"]
    # unequal prime sides where the table's structure does not depend on sizes
    dims = [10] * N if case["equal_dims"] else [5, 7, 11, 13][:N]
    counts = o.schedule_monomial_counts(dims, 3, TREES[case["tree"]], 3)
    want = {(tuple(F), p): c for c, F, p in case["terms"]}
    assert _poly(counts) == want, case["cite"]


def test_standard_tree_per_sweep_tables_1_and_4():
    """Table 1 (N=3) and Table 4 (N=4): item counts of one standard-tree sweep."""
    c3 = o.schedule_monomial_counts([5, 7, 11], 3, o.TREE_STANDARD, 1)
    assert c3 == {((1, 2, 3), 1): 2, ((1, 2), 2): 2, ((1, 3), 2): 1}
    c4 = o.schedule_monomial_counts([5, 7, 11, 13], 3, o.TREE_STANDARD, 1)
    assert c4 == {((1, 2, 3, 4), 1): 2, ((1, 2, 3), 2): 2, ((1, 2), 3): 2, ((1, 3), 3): 1,
                  ((2, 3, 4), 2): 1, ((3, 4), 3): 1}


@pytest.mark.parametrize("tree", ["none", "standard", "restructured"])
def test_corollary1_order5(tree):
    cor = GOLD["corollary1"]
    N = cor["N"]
    counts = o.schedule_monomial_counts([9] * N, 3, TREES[tree], 3)
    got = {"IN_R": 0, "IN1_R2": 0, "I2_RN1": 0}
    for (F, p), c in counts.items():
        if len(F) == N:
            got["IN_R"] += 2 * c
        elif len(F) == N - 1:
            got["IN1_R2"] += 2 * c
        elif len(F) == 2:
            got["I2_RN1"] += 2 * c
    assert got == cor[tree]


def test_restructured_cut_is_one_third_over_three_sweeps_and_half_asymptotically():
    """33% fewer dominant-term flops over three sweeps (Cor. 1); 2(K+1) vs 4K full TTMs over K sweeps."""
    for N in (3, 4, 5):
        dims = [8] * N
        full = {}
        for tree in (o.TREE_STANDARD, o.TREE_RESTRUCTURED):
            s = o.Schedule(dims, 2, tree)
            nfull = []
            for _ in range(50):
                before = len(s.ops)
                ops = s.next_sweep()
                nfull.append(sum(1 for op in ops if op[0] == o.OP_TTM and op[2] == 0))
            full[tree] = nfull
        assert sum(full[o.TREE_RESTRUCTURED][:3]) * 3 == sum(full[o.TREE_STANDARD][:3]) * 2
        assert full[o.TREE_RESTRUCTURED][0] == 2 and all(v == 1 for v in full[o.TREE_RESTRUCTURED][1:])
        assert all(v == 2 for v in full[o.TREE_STANDARD])


@pytest.mark.parametrize("N,tree", [(N, t) for N in (3, 4, 5) for t in (0, 1, 2)])
def test_every_scheduled_leaf_equals_direct_multi_ttm(N, tree):
    """Every update's leaf equals X x_{k != n} Q_k^T with the latest Q_k (brute force),
    over enough sweeps to leave the explicit order-4 sweeps and reach the periodic regime."""
    g = np.random.default_rng(N * 7 + tree)
    dims = [4, 5, 3, 4, 3][:N]
    R = 2
    X = g.standard_normal(dims)
    A0 = [g.standard_normal((d, R)) for d in dims]
    o.cp_als_qr(X, R, A0, tree=tree, extrapolate=True, beta_fixed=0.05, max_sweeps=7, check_leaves=True)


def test_schedule_frees_every_node_it_creates_and_keeps_memory_bounded():
    for N in (3, 4, 5):
        for tree in (0, 1, 2):
            s = o.Schedule([6] * N, 2, tree)
            live_max = 0
            for _ in range(12):
                s.next_sweep()
                live_max = max(live_max, len(s.nodes))
            live = set()
            for op in s.ops:
                if op[0] == o.OP_TTM:
                    live.add(op[1])
                elif op[0] == o.OP_FREE:
                    live.remove(op[1])
            assert live == set(k for k in s.nodes if k != 0)
            assert live_max <= 2 * N


def test_mode_orders():
    s = o.Schedule([10, 10, 10], 3, o.TREE_RESTRUCTURED)
    orders = []
    for _ in range(5):
        orders.append([op[1] + 1 for op in s.next_sweep() if op[0] == o.OP_UPDATE])
    assert orders[0] == [1, 2, 3]
    assert orders[1][0] == 1  # the second sweep starts from the underused Y(1,3) (Section 3.1)
    assert sorted(orders[2]) == [1, 2, 3]
