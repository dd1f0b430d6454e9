"""Pins of the oracle's CP-ALS-QR solver: least-squares equivalences, fit
identities, convergence on exactly low-rank tensors and the beta rule."""
import math

import numpy as np
import pytest

from oracle import cpqr_oracle as o
from paper_2503_18759_gb300 import inputs


def _low_rank(dims, R, seed, eta=0.0):
    B = inputs.gaussian_factors(dims, R, seed)
    X = inputs.add_noise(inputs.cp_dense(B), eta, seed)
    return X, B


@pytest.mark.parametrize("dims,R", [((6, 7, 5), 3), ((4, 5, 3, 4), 2), ((3, 4, 3, 3, 4), 2)])
def test_qr_update_equals_normal_equations_and_lstsq(dims, R):
    """One LS mode update: CP-ALS-QR (Alg. 2) = CP-ALS normal equations (Alg. 1) = lstsq of eq. 6."""
    g = np.random.default_rng(sum(dims))
    X = g.standard_normal(dims)
    A = [g.standard_normal((d, R)) for d in dims]
    for n in range(len(dims)):
        a_qr = o.qr_update_direct(X, A, n)
        a_ne = o.als_normal_update(X, A, n)
        P = o.khatri_rao([A[m] for m in range(len(dims)) if m != n])
        a_ls = np.linalg.lstsq(P, o.unfold(X, n).T, rcond=None)[0].T
        assert np.allclose(a_qr, a_ne, rtol=1e-9, atol=1e-10)
        assert np.allclose(a_qr, a_ls, rtol=1e-10, atol=1e-11)


def test_first_update_of_solver_equals_direct_update():
    g = np.random.default_rng(3)
    dims, R = (5, 6, 4), 3
    X = g.standard_normal(dims)
    A0 = [g.standard_normal((d, R)) for d in dims]
    res = o.cp_als_qr(X, R, A0, tree=o.TREE_STANDARD, extrapolate=False, max_sweeps=1, record=True)
    rec = res.records[0]
    assert rec.mode == 0
    direct = o.qr_update_direct(X, A0, 0)
    assert np.allclose(rec.A * rec.lam, direct, atol=1e-12)


@pytest.mark.parametrize("beta", [0.0, 0.2])
@pytest.mark.parametrize("tree", [o.TREE_NONE, o.TREE_STANDARD, o.TREE_RESTRUCTURED])
def test_reduced_fit_equals_explicit_residual(beta, tree):
    """Section 4.1: ||X||^2 - 2<X,K> + ||K||^2 through V0 and V^ equals the dense residual,
    with and without extrapolation."""
    g = np.random.default_rng(5)
    X, _ = _low_rank((6, 5, 7), 3, 11, eta=0.05)
    A0 = [g.standard_normal((d, 3)) for d in X.shape]
    res = o.cp_als_qr(X, 3, A0, tree=tree, extrapolate=True, beta_schedule=[0.0] + [beta] * 5, max_sweeps=4)
    assert res.fits[-1] == pytest.approx(o.fit_explicit(X, res.lam, res.A), abs=1e-11)


def test_paper_fit_form_r0_rn():
    """Section 4.1: <X,K> = <V, A^ R0^T>, ||K||^2 = <R0^T R0, diag(lam) R_n^T R_n diag(lam)>."""
    g = np.random.default_rng(6)
    X, _ = _low_rank((5, 6, 4), 2, 3, eta=0.1)
    A0 = [g.standard_normal((d, 2)) for d in X.shape]
    res = o.cp_als_qr(X, 2, A0, tree=o.TREE_STANDARD, extrapolate=False, max_sweeps=2, record=True)
    rec = res.records[-1]
    Ahat = rec.A * rec.lam
    inner = float(np.sum(rec.V0 * (Ahat @ rec.R0.T)))
    L = np.diag(rec.lam)
    normK2 = float(np.sum((rec.R0.T @ rec.R0) * (L @ rec.Rn.T @ rec.Rn @ L)))
    fit = 1 - math.sqrt(max(res.normX2 - 2 * inner + normK2, 0)) / math.sqrt(res.normX2)
    assert fit == pytest.approx(res.fits[-1], abs=1e-12)


@pytest.mark.parametrize("tree", [o.TREE_STANDARD, o.TREE_RESTRUCTURED])
@pytest.mark.parametrize("dims,R", [((12, 10, 11), 3), ((7, 8, 6, 7), 2)])
def test_exact_low_rank_converges_to_fit_one(tree, dims, R):
    """ALS-QR(-BR) on an exactly rank-R tensor from known factors: fit -> 1 and the
    factors are recovered up to permutation and scale."""
    X, B = _low_rank(dims, R, 21)
    A0 = inputs.init_factors(dims, R, 22)
    res = o.cp_als_qr(X, R, A0, tree=tree, extrapolate=False, max_sweeps=400, tol=1e-15)
    assert res.fits[-1] > 1 - 1e-7
    assert o.fit_explicit(X, res.lam, res.A) > 1 - 1e-7
    assert o.factor_match_score(B, res.A) > 0.9999


@pytest.mark.parametrize("beta", [1 / 250, 1 / 2000])
def test_extrapolated_fixed_point_is_scaled_by_one_plus_beta_one_minus_alpha(beta):
    """At a fixed point Q0^k = Q0^{k-1}, eq. 19 gives Q0^ = (1 + beta (1 - alpha)) Q0, so on an
    exactly low-rank tensor the model is the exact tensor scaled by that factor and the fit
    settles at 1 - beta (1 - alpha)."""
    X, B = _low_rank((12, 10, 11), 3, 21)
    A0 = inputs.init_factors(X.shape, 3, 22)
    res = o.cp_als_qr(X, 3, A0, tree=o.TREE_RESTRUCTURED, extrapolate=True, beta_fixed=beta,
                      max_sweeps=400, tol=1e-15)
    assert res.fits[-1] == pytest.approx(1 - beta * (1 - o.ALPHA), abs=1e-9)
    assert o.factor_match_score(B, res.A) > 0.9999


def test_beta_zero_reproduces_br_bit_for_bit():
    g = np.random.default_rng(8)
    X, _ = _low_rank((6, 7, 5), 3, 4, eta=0.01)
    A0 = [g.standard_normal((d, 3)) for d in X.shape]
    a = o.cp_als_qr(X, 3, A0, tree=o.TREE_RESTRUCTURED, extrapolate=False, max_sweeps=6)
    b = o.cp_als_qr(X, 3, A0, tree=o.TREE_RESTRUCTURED, extrapolate=True, beta_fixed=0.0, max_sweeps=6)
    assert a.fits == b.fits
    for x, y in zip(a.A, b.A):
        assert np.array_equal(x, y)


def test_tree_choice_does_not_change_the_iterates_when_order_is_the_same():
    """Standard tree and no tree update modes in the same order 1..N: identical iterates
    up to rounding (the tree only reorders the TTMs)."""
    g = np.random.default_rng(9)
    X, _ = _low_rank((6, 5, 7, 4), 2, 5, eta=0.02)
    A0 = [g.standard_normal((d, 2)) for d in X.shape]
    a = o.cp_als_qr(X, 2, A0, tree=o.TREE_NONE, extrapolate=False, max_sweeps=5)
    b = o.cp_als_qr(X, 2, A0, tree=o.TREE_STANDARD, extrapolate=False, max_sweeps=5)
    assert np.allclose(a.fits, b.fits, atol=1e-12)


def test_beta_rule_bands_and_activation():
    """Section 4.2: alpha = 1/10; beta picked once |fit_k - fit_{k-1}| < 0.03 by fit level."""
    assert o.ALPHA == 0.1
    assert o.beta_band(0.99) == 1 / 20000 and o.beta_band(0.951) == 1 / 20000
    assert o.beta_band(0.95) == 1 / 2000 and o.beta_band(0.91) == 1 / 2000
    assert o.beta_band(0.90) == 1 / 500 and o.beta_band(0.75) == 1 / 500
    assert o.beta_band(0.70) == 1 / 250 and o.beta_band(0.2) == 1 / 250
    r = o.BetaRule()
    assert r.observe(0.5) == 0.0          # sweep 1: nothing to compare with
    assert r.observe(0.6) == 0.0          # change 0.1 >= 0.03: stays off
    assert r.observe(0.62) == 1 / 250     # change 0.02: activates at fit 0.62
    assert r.activated_after == 3
    assert r.observe(0.97) == 1 / 250     # fixed once chosen
    r2 = o.BetaRule()
    r2.observe(0.955)
    assert r2.observe(0.96) == 1 / 20000


def test_solver_applies_beta_from_the_sweep_after_activation():
    g = np.random.default_rng(10)
    X, _ = _low_rank((8, 7, 9), 3, 6, eta=0.05)
    A0 = [g.standard_normal((d, 3)) for d in X.shape]
    res = o.cp_als_qr(X, 3, A0, tree=o.TREE_RESTRUCTURED, extrapolate=True, max_sweeps=12)
    rule = o.BetaRule()
    expect = [0.0]
    for f in res.fits[:-1]:
        expect.append(rule.observe(f))
    assert res.betas == expect


def test_generator_collinear_factors_have_exact_congruence():
    """Section 4.2 construction: unit columns with pairwise cosine exactly c."""
    for c in (0.0, 0.5, 0.9):
        B = inputs.collinear_factors([40, 30], 6, c, seed=3)
        for b in B:
            G = b.T @ b
            assert np.allclose(np.diag(G), 1, atol=1e-13)
            off = G[~np.eye(6, dtype=bool)]
            assert np.allclose(off, c, atol=1e-13)


def test_generator_noise_level():
    X = inputs.cp_dense(inputs.gaussian_factors([10, 11, 12], 3, 1))
    Y = inputs.add_noise(X, 1e-3, 1)
    assert np.linalg.norm((Y - X).ravel()) / np.linalg.norm(X.ravel()) == pytest.approx(1e-3, rel=1e-12)
    assert inputs.eta_from_l1(0.01) == pytest.approx(1 / math.sqrt(100 / 0.01 - 1))
