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


def _corollary1_terms(N, tree):
    counts = o.schedule_monomial_counts([9] * N, 3, TREES[tree], 3)
    got = {"IN_R": 0, "IN1_R2": 0, "I2_RN1": 0}
    for (F, p), c in counts.items():
        if len(F) == N:
            got["IN_R"] += 2 * c
        elif len(F) == N - 1:
            got["IN1_R2"] += 2 * c
        elif len(F) == 2:
            got["I2_RN1"] += 2 * c
    return got


@pytest.mark.parametrize("tree", ["none", "standard", "restructured"])
def test_corollary1_order5(tree):
    cor = GOLD["corollary1"]
    assert _corollary1_terms(cor["N"], tree) == cor[tree]


@pytest.mark.parametrize("tree", ["none", "standard", "restructured"])
def test_corollary1_order6(tree):
    """Corollary 1 holds for every order N > 4: over the first three sweeps the coefficients of
    I^N R, I^(N-1) R^2 and I^2 R^(N-1) are 6N, 6N, 6N (no tree), 12, 18, 6N (dimension tree) and
    8, 14, 6N (restructured tree).  At N = 6: 36, 36, 36 / 12, 18, 36 / 8, 14, 36."""
    N = 6
    want = {"none": {"IN_R": 6 * N, "IN1_R2": 6 * N, "I2_RN1": 6 * N},
            "standard": {"IN_R": 12, "IN1_R2": 18, "I2_RN1": 6 * N},
            "restructured": {"IN_R": 8, "IN1_R2": 14, "I2_RN1": 6 * N}}
    assert _corollary1_terms(N, tree) == want[tree]


def test_restructured_cut_is_one_third_over_three_sweeps_and_half_asymptotically():
    """33% fewer dominant-term flops over three sweeps (Cor. 1); 2(K+1) vs 4K full TTMs over K sweeps."""
    for N in (3, 4, 5, 6):
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


@pytest.mark.parametrize("N,tree", [(N, t) for N in (3, 4, 5, 6) for t in (0, 1, 2)])
def test_every_scheduled_leaf_equals_direct_multi_ttm(N, tree):
    """Every update's leaf equals X x_{k != n} Q_k^T with the latest Q_k (brute force),
    over enough sweeps to leave the explicit order-4 sweeps and reach the periodic regime."""
    g = np.random.default_rng(N * 7 + tree)
    dims = [4, 5, 3, 4, 3, 3][:N]
    R = 2
    X = g.standard_normal(dims)
    A0 = [g.standard_normal((d, R)) for d in dims]
    o.cp_als_qr(X, R, A0, tree=tree, extrapolate=True, beta_fixed=0.05, max_sweeps=7, check_leaves=True)


def test_schedule_frees_every_node_it_creates_and_keeps_memory_bounded():
    for N in (3, 4, 5, 6):
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


def test_mode_orders_order3_follow_section_3_1():
    """Order 3 (Section 3.1): sweep 2 starts from the unused Y(1,3) to update A1 and forms Y(2,3)
    from X for A2 and A3; sweep 3 proceeds from Y(2,3) (A2) and forms Y(1,3) from X for A1 and A3;
    sweeps 4, 5, ... repeat them."""
    s = o.Schedule([10, 10, 10], 3, o.TREE_RESTRUCTURED)
    orders, sources = [], []
    free_of = {0: (0, 1, 2)}
    for _ in range(6):
        ops = s.next_sweep()
        orders.append([op[1] + 1 for op in ops if op[0] == o.OP_UPDATE])
        first_src = None
        for op in ops:
            if op[0] == o.OP_TTM:
                free_of[op[1]] = tuple(m for m in free_of[op[2]] if m != op[3])
                if first_src is None:
                    first_src = tuple(m + 1 for m in free_of[op[2]])
        sources.append(first_src)
    assert orders == [[1, 2, 3], [1, 2, 3], [2, 1, 3], [1, 2, 3], [2, 1, 3], [1, 2, 3]]
    assert sources[1:4] == [(1, 3), (2, 3), (1, 3)]


@pytest.mark.parametrize("N", [3, 4, 5, 6])
@pytest.mark.parametrize("tree", [o.TREE_NONE, o.TREE_STANDARD, o.TREE_RESTRUCTURED])
def test_every_sweep_updates_each_mode_once_and_no_update_is_a_no_op(N, tree):
    """Alternating updates (Section 3.1): each sweep updates every mode exactly once, and no update
    repeats the mode updated just before it (that update would see no changed factor: the same
    leaf, the same Khatri-Rao QR, the same least-squares solution)."""
    s = o.Schedule([7] * N, 3, tree)
    ups = []
    for _ in range(50):
        modes = [op[1] for op in s.next_sweep() if op[0] == o.OP_UPDATE]
        assert sorted(modes) == list(range(N))
        ups += modes
    assert all(ups[j] != ups[j - 1] for j in range(1, len(ups))), ups


@pytest.mark.parametrize("c,seed", [(0.3, 0), (0.3, 1), (0.5, 0), (0.5, 1)])
def test_restructured_tree_converges_in_about_the_standard_trees_sweeps(c, seed):
    """Without extrapolation both trees take exact least-squares steps and reach the same fit.
    The restructured tree updates some modes after only one other factor changed (its order,
    Section 3.1), so it needs a few more sweeps than the standard tree (1.1-1.2x on these
    problems), never the ~1.5x that one wasted update per sweep costs."""
    from paper_2503_18759_gb300 import inputs
    p = inputs.make_problem("conv", [30, 30, 30], 6, seed=seed, c=c, eta=1e-3, dtype=np.float64)
    std = o.cp_als_qr(p.X, 6, p.A0, tree=o.TREE_STANDARD, extrapolate=False, max_sweeps=90).fits
    res = o.cp_als_qr(p.X, 6, p.A0, tree=o.TREE_RESTRUCTURED, extrapolate=False, max_sweeps=90).fits
    target = max(std) - 1e-6
    k_std = next(i for i, f in enumerate(std) if f >= target) + 1
    k_res = next(i for i, f in enumerate(res) if f >= target) + 1
    assert abs(max(res) - max(std)) < 1e-9
    assert k_res <= 1.3 * k_std, (k_std, k_res)
    assert all(b >= a - 1e-12 for a, b in zip(res, res[1:]))  # exact LS steps: the fit never drops
