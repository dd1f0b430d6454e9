"""The slab partition of CP-ALS-QR across ranks, simulated on CPU ranks (gloo, world size 2).

Each rank holds the slab X[rows_r, ...] of the partitioned mode p = 0 (the slowest index in C
order) and runs the same schedule on it.  Every contraction is linear, so:
* an intermediate that contracted mode p holds this rank's partial sum, one that did not holds
  this rank's rows of mode p;
* the update of a mode n != p needs V_n = Y_(n) [Q0 | Q0^{k-1}] (I_n x 2R) summed over the
  ranks: one all-reduce, after which the solve, the normalisation and the factor QR are
  replicated;
* the update of mode p keeps its rows local: V_p, the solve and A^ are row slices; the column
  norms come from an all-reduce of squared norms, and the QR of A^(p) is a TSQR (local QR, an
  all-gather of the R x R triangles, a QR of their stack, Q_r = A_r R^{-1});
* ||X||^2 and the fit terms of a mode-p update are all-reduced; the Khatri-Rao QRs (of the
  replicated triangles R_k) are replicated.
The result must equal the single-process oracle's to rounding (the sums only change order)."""
import math
import os
import socket

import numpy as np
import pytest

from oracle import cpqr_oracle as o

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _rows(I, rank, world):
    lo = rank * I // world
    hi = (rank + 1) * I // world
    return lo, hi


def _allreduce(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
    dist.all_reduce(t)
    return t.numpy()


def _allgather(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
    out = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(out, t)
    return [x.numpy() for x in out]


def _allgather_rows(a, I):
    """Stack every rank's row slice of an I-row matrix (slices padded to equal size for gloo)."""
    world = dist.get_world_size()
    width = -(-I // world)
    pad = np.zeros((width, a.shape[1]))
    pad[:a.shape[0]] = a
    parts = _allgather(pad)
    return np.vstack([parts[r][:_rows(I, r, world)[1] - _rows(I, r, world)[0]] for r in range(world)])


def partitioned_cp_als_qr(X_slab, dims, rows, R, A0, tree, beta_fixed, sweeps, p=0):
    """CP-ALS-QR (Alg. 2 / 3 with a fixed beta from the second sweep) on this rank's slab of mode p."""
    N = len(dims)
    lo, hi = rows
    normX2 = float(_allreduce(np.array([np.sum(X_slab * X_slab)]))[0])
    A = [np.asarray(a, dtype=np.float64).copy() for a in A0]
    Q, Rf = [], []
    for a in A:
        q, r = o.householder_qr(a)
        Q.append(q)
        Rf.append(r)
    Q0prev = [None] * N
    sched = o.Schedule(dims, R, tree)
    store = {0: X_slab}
    partial = {0: False}  # whether a node holds a partial sum over the ranks (mode p contracted)
    fits = []
    lam = np.ones(R)
    for k in range(sweeps):
        beta = beta_fixed if k >= 1 else 0.0
        last = None
        for op in sched.next_sweep():
            if op[0] == o.OP_TTM:
                _, dst, src, m = op
                Qm = Q[m][lo:hi] if m == p else Q[m]
                store[dst] = o.ttm_qt(store[src], Qm, m)
                partial[dst] = partial[src] or m == p
            elif op[0] == o.OP_FREE:
                store.pop(op[1], None)
            else:
                _, n, leaf, _ = op
                Z = o.khatri_rao([Rf[m] for m in range(N) if m != n])
                Q0, R0 = o.householder_qr(Z)
                Q0hat = o.extrapolate_q0(Q0, Q0prev[n], beta, o.ALPHA) if (beta and Q0prev[n] is not None) else Q0
                Yn = o.unfold(store[leaf], n)
                V0, Vhat = Yn @ Q0, Yn @ Q0hat
                if n != p:
                    assert partial[leaf]
                    V = _allreduce(np.concatenate([V0, Vhat], axis=1))
                    V0, Vhat = V[:, :R], V[:, R:]
                    Ahat = o.solve_upper_transposed(Vhat, R0)
                    lam = np.linalg.norm(Ahat, axis=0)
                    A[n] = Ahat / lam[None, :]
                    Q[n], Rf[n] = o.householder_qr(A[n])
                    terms = np.array([np.sum(V0 * Vhat), np.sum(Vhat * Vhat)])
                else:
                    assert not partial[leaf]  # rows lo:hi of mode p
                    Ahat_r = o.solve_upper_transposed(Vhat, R0)
                    lam = np.sqrt(_allreduce(np.sum(Ahat_r * Ahat_r, axis=0)))
                    A_r = Ahat_r / lam[None, :]
                    # TSQR: local triangles (a slab shorter than R padded with zero rows), the QR of
                    # their stack, then Q_r = A_r R^{-1}
                    pad = np.zeros((max(R - A_r.shape[0], 0), R))
                    _, Rr = o.householder_qr(np.vstack([A_r, pad]))
                    _, Rp = o.householder_qr(np.vstack(_allgather(Rr)))
                    Q_r = np.linalg.solve(Rp.T, A_r.T).T
                    A[n] = _allgather_rows(A_r, dims[p])
                    Q[n] = _allgather_rows(Q_r, dims[p])
                    Rf[n] = Rp
                    terms = _allreduce(np.array([np.sum(V0 * Vhat), np.sum(Vhat * Vhat)]))
                Q0prev[n] = Q0
                last = terms
        res2 = normX2 - 2.0 * last[0] + last[1]
        fits.append(1.0 - math.sqrt(max(res2, 0.0)) / math.sqrt(normX2))
    return A, lam, fits


def _worker(rank, world, port, case, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, dims, R, A0, tree, beta, sweeps = case
        lo, hi = _rows(dims[0], rank, world)
        A, lam, fits = partitioned_cp_als_qr(X[lo:hi], dims, (lo, hi), R, A0, tree, beta, sweeps)
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), fits=np.array(fits), lam=lam, *A)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("dims,R,tree,beta", [([9, 8, 7], 3, o.TREE_RESTRUCTURED, 0.02),
                                             ([7, 6, 5, 6], 2, o.TREE_STANDARD, 0.0),
                                             ([6, 5, 4, 5, 4], 2, o.TREE_RESTRUCTURED, 0.01)])
def test_slab_partition_on_two_gloo_ranks_matches_the_oracle(tmp_path, dims, R, tree, beta):
    from paper_2503_18759_gb300 import inputs
    B = inputs.gaussian_factors(dims, R, 3)
    X = inputs.add_noise(inputs.cp_dense(B), 1e-3, 3)
    A0 = inputs.init_factors(dims, R, 3)
    sweeps = 5
    case = (X, dims, R, A0, tree, beta, sweeps)
    world = 2
    torch.multiprocessing.spawn(_worker, args=(world, _free_port(), case, str(tmp_path)), nprocs=world, join=True)
    kw = dict(extrapolate=beta > 0, beta_fixed=beta if beta > 0 else None)
    ref = o.cp_als_qr(X, R, A0, tree=tree, max_sweeps=sweeps, **kw)
    for rank in range(world):
        d = np.load(os.path.join(tmp_path, f"r{rank}.npz"))
        assert np.allclose(d["fits"], ref.fits, rtol=0, atol=1e-12), (d["fits"], ref.fits)
        assert np.allclose(d["lam"], ref.lam, rtol=1e-11)
        for n in range(len(dims)):
            assert np.allclose(d[f"arr_{n}"], ref.A[n], atol=1e-10), n
