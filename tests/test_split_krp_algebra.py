"""Host restatement of the split Khatri-Rao QR and of the structure-aware assembly
(csrc/krp_gram.cu::launch_krp_rows_split, csrc/smallqr.cu::krp_assemble_tri_kernel).

The QR of Z = R_1 (.) ... (.) R_m (Alg. 3, lines 3-4: the Khatri-Rao product of the factors'
triangles, row index (i_1, ..., i_m) with i_m fastest) is assembled from the QR of W, the product
of all triangles but the one at position s, and the QR of the two-triangle product
Y = R_s (.) S_W: Q0[(l, i, t)] = sum_j Q_W[(l, t), j] Q_Y[(i, j)] with l over the triangles
before s and t over those after, R0 = R_Y.  These tests pin the row mapping against the direct
Householder QR of Z, the exact zeros of Q_Y that the structure-aware assembly skips, and the
integer rule that splits a row's columns into parts of equal cost."""
import numpy as np
import pytest

from oracle import cpqr_oracle as o


def _triangles(m, R, seed):
    g = np.random.default_rng(seed)
    return [o.householder_qr(g.standard_normal((R + 3, R)))[1] for _ in range(m)]


def _split_qr(tri, s):
    m, R = len(tri), tri[0].shape[0]
    W = o.khatri_rao([t for k, t in enumerate(tri) if k != s])
    QW, SW = o.householder_qr(W)
    QY, RY = o.householder_qr(o.khatri_rao([tri[s], SW]))
    L, T = R ** s, R ** (m - 1 - s)
    # Q0[(l, i, t), c] = sum_j QW[(l, t), j] QY[(i, j), c]
    Q0 = np.einsum("ltj,ijc->litc", QW.reshape(L, T, R), QY.reshape(R, R, R)).reshape(L * R * T, R)
    return Q0, RY


@pytest.mark.parametrize("m,R", [(3, 3), (3, 5), (4, 3), (4, 4)])
def test_split_route_gives_the_qr_of_the_product(m, R):
    tri = _triangles(m, R, 10 * m + R)
    Z = o.khatri_rao(tri)
    Qr, Rr = o.householder_qr(Z)
    for s in range(m):
        Q0, R0 = _split_qr(tri, s)
        assert np.abs(Q0.T @ Q0 - np.eye(R)).max() < 1e-14
        assert np.allclose(R0, Rr, atol=1e-13 * np.abs(Rr).max()), s
        assert np.allclose(Q0, Qr, atol=1e-13), s


def test_a_wrong_row_mapping_is_caught():
    """Planted mistake: assembling with (i, l, t) instead of (l, i, t) must not pass."""
    m, R, s = 3, 4, 1
    tri = _triangles(m, R, 7)
    Qr, _ = o.householder_qr(o.khatri_rao(tri))
    W = o.khatri_rao([t for k, t in enumerate(tri) if k != s])
    QW, SW = o.householder_qr(W)
    QY, _ = o.householder_qr(o.khatri_rao([tri[s], SW]))
    L, T = R ** s, R ** (m - 1 - s)
    bad = np.einsum("ltj,ijc->iltc", QW.reshape(L, T, R), QY.reshape(R, R, R)).reshape(-1, R)
    assert not np.allclose(bad, Qr, atol=1e-6)


def _forward_substitution(Y, R1):
    """q R1 = y row by row, column by column (the rows kernels' order)."""
    Q = np.zeros_like(Y)
    for r in range(Y.shape[0]):
        x = Y[r].copy()
        for c in range(Y.shape[1]):
            x[c] = x[c] / R1[c, c]
            x[c + 1:] -= x[c] * R1[c, c + 1:]
        Q[r] = x
    return Q


def test_gram_route_rows_keep_the_staircase_zeros_exactly():
    """Row (i, j) of Y = R_a (.) S is zero left of column max(i, j), and a forward substitution
    against an upper triangle (Q1 = Y R1^{-1}) keeps those entries exactly zero: the
    structure-aware assembly may skip them without changing a single result."""
    R = 6
    Ra, S = _triangles(2, R, 3)
    Y = o.khatri_rao([Ra, S])
    R1 = np.linalg.cholesky(Y.T @ Y).T
    Q1 = _forward_substitution(Y, R1)
    for i in range(R):
        for j in range(R):
            row = Q1[i * R + j]
            assert np.all(row[:max(i, j)] == 0.0)
    assert np.abs(Q1.T @ Q1 - np.eye(R)).max() < 1e-13


def test_skipping_the_zeros_changes_no_bit():
    """The dense sum over j and the kept terms j <= c (c >= i), in the same order, agree bit for
    bit (up to the sign of zero) when Q_Y has the staircase zeros."""
    R, LT = 5, 7
    g = np.random.default_rng(1)
    QW = g.standard_normal((LT, R))
    QY = g.standard_normal((R, R, R))
    for i in range(R):
        for j in range(R):
            QY[i, j, :max(i, j)] = 0.0
    for w in range(LT):
        for i in range(R):
            for c in range(R):
                dense = 0.0
                for j in range(R):
                    dense = dense + QW[w, j] * QY[i, j, c]
                kept = 0.0
                if c >= i:
                    for j in range(c + 1):
                        kept = kept + QW[w, j] * QY[i, j, c]
                assert dense == kept


def _owner_parts(R, i, P):
    """The kernel's rule: column c >= i costs c + 1 and starts at (c (c+1) - i (i+1)) / 2 of the
    row's total; it belongs to part k when k * total <= start * P < (k + 1) * total (the last
    part takes the rest); the zero columns c < i belong to part 0."""
    total = (R * (R + 1) - i * (i + 1)) // 2
    owners = []
    for c in range(R):
        if c < i:
            owners.append([0])
            continue
        sp = (c * (c + 1) - i * (i + 1)) // 2 * P
        owners.append([k for k in range(P) if sp >= k * total and (k == P - 1 or sp < (k + 1) * total)])
    return owners, total


@pytest.mark.parametrize("R", [1, 2, 3, 5, 8, 16, 17, 24, 32])
def test_column_parts_cover_every_column_once(R):
    for P in range(1, max(1, R // 2) + 1):
        for i in range(R):
            owners, total = _owner_parts(R, i, P)
            assert all(len(ow) == 1 for ow in owners), (R, P, i)
            seq = [ow[0] for ow in owners]
            assert seq == sorted(seq)  # contiguous ranges
            cost = [0] * P
            for c in range(i, R):
                cost[seq[c]] += c + 1
            assert sum(cost) == total
            # no part exceeds its share by more than one column's cost
            assert max(cost) <= total / P + R


@pytest.mark.parametrize("dims", [[9, 8, 7], [7, 6, 5, 6], [5, 4, 5, 4, 5]])
def test_no_update_repeats_the_khatri_rao_qr_of_the_update_before_it(dims):
    """No update repeats the mode of the update before it (alternating updates, Section 3.1), so
    every update's Khatri-Rao QR (Alg. 3, lines 3-4) has a changed triangle and differs from the
    previous one; the library's schedule gives the oracle's update order."""
    from paper_2503_18759_gb300 import inputs
    R, sweeps = 3, 6
    B = inputs.gaussian_factors(dims, R, 2)
    X = inputs.add_noise(inputs.cp_dense(B), 1e-3, 2)
    res = o.cp_als_qr(X, R, inputs.init_factors(dims, R, 2), tree=o.TREE_RESTRUCTURED, max_sweeps=sweeps,
                      beta_fixed=0.05, record=True)
    recs = res.records
    for a, c in zip(recs, recs[1:]):
        assert a.mode != c.mode
        assert not np.array_equal(a.R0, c.R0)
    from paper_2503_18759_gb300 import binding as b
    ops, _ = b.cp_als_qr_schedule(dims, R, b.TREE_RESTRUCTURED, sweeps)
    assert [r.mode for r in recs] == [int(op[1]) for op in ops if int(op[0]) == 1]
