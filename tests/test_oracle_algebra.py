"""Pins of the oracle's tensor algebra and QR against definitions that do not
go through the oracle's own code paths (brute force, closed forms, numpy)."""
import itertools

import numpy as np
import pytest

from oracle import cpqr_oracle as o


def _rng(s=0):
    return np.random.default_rng(s)


@pytest.mark.parametrize("shape", [(3, 4, 5), (2, 3, 4, 3), (2, 2, 3, 2, 2)])
def test_mode_product_brute_force(shape):
    """Section 2.1 definition of the mode-n product, summed element by element."""
    g = _rng(1)
    T = g.standard_normal(shape)
    for n in range(len(shape)):
        B = g.standard_normal((2, shape[n]))
        Y = o.mode_product(T, B, n)
        out_shape = list(shape)
        out_shape[n] = 2
        assert Y.shape == tuple(out_shape)
        for idx in itertools.product(*[range(s) for s in out_shape]):
            acc = 0.0
            for i in range(shape[n]):
                src = list(idx)
                src[n] = i
                acc += T[tuple(src)] * B[idx[n], i]
            assert abs(Y[idx] - acc) < 1e-12


def test_kron_matches_numpy():
    g = _rng(2)
    A, B = g.standard_normal((3, 2)), g.standard_normal((4, 5))
    assert np.allclose(o.kron(A, B), np.kron(A, B), atol=0, rtol=0)


def test_khatri_rao_columns_are_kronecker():
    g = _rng(3)
    A, B, C = g.standard_normal((3, 4)), g.standard_normal((2, 4)), g.standard_normal((5, 4))
    K = o.khatri_rao([A, B, C])
    for r in range(4):
        assert np.allclose(K[:, r], np.kron(A[:, r], np.kron(B[:, r], C[:, r])), atol=1e-15)


def test_eq1_mixed_product():
    """(C (x) D)(A (.) B) = (CA) (.) (DB)  (eq. 1)."""
    g = _rng(4)
    A, B = g.standard_normal((3, 4)), g.standard_normal((5, 4))
    C, D = g.standard_normal((2, 3)), g.standard_normal((6, 5))
    lhs = np.kron(C, D) @ o.khatri_rao([A, B])
    rhs = o.khatri_rao([C @ A, D @ B])
    assert np.allclose(lhs, rhs, atol=1e-12)


@pytest.mark.parametrize("shape", [(3, 4, 5), (2, 3, 4, 3)])
def test_eq3_multi_ttm_unfolding(shape):
    """Multi-TTM over every mode but n: Y_(n) = X_(n) (B_N (x) ... (x) B_{n+1} (x) B_{n-1} (x) ... (x) B_1)^T
    in the paper's (first-index-fastest) unfolding, eq. 3 (printed with n-1 and n+1 swapped);
    and the C-order analogue used by the build."""
    g = _rng(5)
    X = g.standard_normal(shape)
    N = len(shape)
    Bs = [g.standard_normal((2 + k % 2, s)) for k, s in enumerate(shape)]
    for n in range(N):
        Y = X
        for k, B in enumerate(Bs):
            if k != n:
                Y = o.mode_product(Y, B, k)
        others_desc = [Bs[k] for k in range(N - 1, -1, -1) if k != n]
        K = others_desc[0]
        for B in others_desc[1:]:
            K = np.kron(K, B)
        assert np.allclose(o.unfold_kolda(Y, n), o.unfold_kolda(X, n) @ K.T, atol=1e-11)
        others_asc = [Bs[k] for k in range(N) if k != n]
        K = others_asc[0]
        for B in others_asc[1:]:
            K = np.kron(K, B)
        assert np.allclose(o.unfold(Y, n), o.unfold(X, n) @ K.T, atol=1e-11)


@pytest.mark.parametrize("m,n", [(7, 3), (40, 5), (64, 32), (5, 5), (400, 32)])
def test_householder_qr_properties(m, n):
    g = _rng(m * 100 + n)
    A = g.standard_normal((m, n))
    Q, R = o.householder_qr(A)
    assert Q.shape == (m, n) and R.shape == (n, n)
    assert np.allclose(Q.T @ Q, np.eye(n), atol=1e-13)
    assert np.allclose(Q @ R, A, atol=1e-12 * np.linalg.norm(A))
    assert np.all(np.tril(R, -1) == 0)
    assert np.all(np.diag(R) > 0)
    # uniqueness: equals LAPACK's QR after normalising its signs
    q2, r2 = np.linalg.qr(A)
    d = np.sign(np.diag(r2))
    assert np.allclose(Q, q2 * d, atol=1e-12)
    assert np.allclose(R, r2 * d[:, None], atol=1e-11 * np.linalg.norm(A))


def test_householder_qr_handles_negative_pivots():
    A = np.array([[-3.0, 1.0], [4.0, 2.0], [0.0, -1.0]])
    Q, R = o.householder_qr(A)
    assert R[0, 0] == pytest.approx(5.0)
    assert np.all(np.diag(R) > 0)
    assert np.allclose(Q @ R, A, atol=1e-14)


@pytest.mark.parametrize("N,R", [(3, 4), (4, 3), (5, 2)])
def test_q0_first_row_and_column_are_e1(N, R):
    """Section 3.2: Q0 from the KRP of triangular R_k has e1 as first row and column."""
    g = _rng(N * 10 + R)
    Rs = []
    for _ in range(N - 1):
        _, r = o.householder_qr(g.standard_normal((R + 3, R)))
        Rs.append(r)
    Z = o.khatri_rao(Rs)
    Q0, R0 = o.householder_qr(Z)
    e1 = np.zeros(R)
    e1[0] = 1
    assert np.allclose(Q0[0, :], e1, atol=1e-14)
    e1c = np.zeros(Z.shape[0])
    e1c[0] = 1
    assert np.allclose(Q0[:, 0], e1c, atol=1e-14)
    assert np.allclose(Q0.T @ Q0, np.eye(R), atol=1e-13)
    assert np.allclose(Q0 @ R0, Z, atol=1e-12)


def test_eq18_keeps_e1_structure_eq19_scales_it():
    """Section 3.2: plain extrapolation (eq. 18, alpha = 1) leaves the first row and column
    of Q0 untouched; the customised form (eq. 19) scales them by 1 + beta (1 - alpha)."""
    g = _rng(9)
    mats = []
    for s in range(2):
        Rs = [o.householder_qr(g.standard_normal((6, 3)))[1] for _ in range(2)]
        mats.append(o.householder_qr(o.khatri_rao(Rs))[0])
    Q0, Q0prev = mats
    beta = 0.3
    q18 = o.extrapolate_q0(Q0, Q0prev, beta, 1.0)
    assert q18[0, 0] == pytest.approx(1.0, abs=1e-14)
    assert np.allclose(q18[0, 1:], 0, atol=1e-14) and np.allclose(q18[1:, 0], 0, atol=1e-14)
    q19 = o.extrapolate_q0(Q0, Q0prev, beta, 0.1)
    assert q19[0, 0] == pytest.approx(1.0 + beta * 0.9, abs=1e-14)
    # off the first row/column both forms agree with the definition entrywise
    assert np.allclose(q19[1:, 1:], Q0[1:, 1:] + beta * (Q0[1:, 1:] - 0.1 * Q0prev[1:, 1:]), atol=1e-15)


def test_solve_upper_transposed_back_substitution():
    g = _rng(11)
    R0 = np.triu(g.standard_normal((5, 5))) + 3 * np.eye(5)
    V = g.standard_normal((7, 5))
    A = o.solve_upper_transposed(V, R0)
    assert np.allclose(A @ R0.T, V, atol=1e-12)


def test_cp_full_matches_outer_products():
    g = _rng(12)
    A = [g.standard_normal((3, 2)), g.standard_normal((4, 2)), g.standard_normal((2, 2))]
    lam = np.array([2.0, -0.5])
    K = o.cp_full(lam, A)
    for i, j, k in itertools.product(range(3), range(4), range(2)):
        ref = sum(lam[r] * A[0][i, r] * A[1][j, r] * A[2][k, r] for r in range(2))
        assert abs(K[i, j, k] - ref) < 1e-13
