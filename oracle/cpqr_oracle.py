"""FP64 CPU oracle for CP-ALS-QR, ALS-QR-BR and ALS-QR-BRE.

TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.  Only the test suite, the
``smoke()`` check and the CPU-baseline leg of the benchmark may import this
module.  The CUDA library never calls it and shares no code with it.

It restates, step by step and in float64, what the paper defines:

* mode-n product / TTM and its unfolding identity (Section 2.1, eq. 3),
  Khatri-Rao / Kronecker mixed product (eq. 1);
* the CP-ALS-QR mode update (Alg. 2): Z_n = KRP of the R_k, Z_n = Q0 R0,
  Y = X x_{k != n} Q_k^T, V = Y_(n) Q0, solve A^ R0^T = V, normalise, QR;
* the customised extrapolation on Q0 (eq. 19, Alg. 3) and the beta / alpha
  rule of Section 4.2;
* the TTM schedules: no tree, the standard dimension tree and the
  restructured dimension tree (Section 3.1, Tables 1-6, Cor. 1) with an
  exact flop counter (cost 2 * R * prod(source dims) per TTM, Section 3.4);
* the approximation error / fitness of Section 4.1.

Readings of the paper where it is silent or garbled (all restated in the
design notes of the repository):

* Storage is C order (last index fastest).  Unfoldings flatten the remaining
  indices in C order, so Z_n lists its rows (r_1..r_N without r_n) with the
  last index fastest, matching the columns of Y_(n).
* Every QR is normalised to a positive diagonal of R; this makes Q0 unique,
  gives Q0[0,0] = 1 (the structure noted in Section 3.2) and makes eq. 19's
  difference Q0^k - alpha Q0^{k-1} meaningful.
* Q0^{k-1} is the unextrapolated Q0 of the same mode in the previous sweep.
* Stopping: "fitness >= eps" in Alg. 2/3 is read as |fit_k - fit_{k-1}| < tol.
* Fit after the last mode of a sweep: ||X-K||^2 = ||X||^2 - 2<V0, V^> + ||V^||^2
  with V0 = Y_(n) Q0 and V^ = Y_(n) Q0^ (exact under extrapolation; equal to
  ||X||^2 - ||V0||^2 without it and to Section 4.1's R0/R_n form).
* beta rule (Section 4.2): checked after every sweep k >= 2 until active;
  activates when |fit_k - fit_{k-1}| < 0.03 with beta = 1/20000 (fit > 0.95),
  1/2000 (0.90 < fit <= 0.95), 1/500 (0.70 < fit <= 0.90), else 1/250; alpha =
  1/10; beta then stays fixed and applies from sweep k+1.
* Restructured tree: sweep 1 is the standard tree.  Order 3 then alternates
  the two sweeps Section 3.1 describes: sweep 2 starts from the unused
  Y(1,3) (A1) and forms Y(2,3) from X (A2, A3); sweep 3 proceeds from Y(2,3)
  (A2) and forms Y(1,3) from X (A1, A3); sweeps 4, 5, ... repeat them.  For
  order 4, sweeps 2 and 3 follow the structure that Table 5 counts.  Every
  other sweep picks, among the modes not yet updated in the sweep and whose
  update would not be a no-op (an update is a no-op when no other factor
  changed since that mode's last update: same leaf, same Khatri-Rao QR, same
  result), the cheapest valid cached source (ties: lowest mode), and
  contracts first the modes already updated in this sweep, then ascending.
  Every update thus follows a change of another factor (the alternating
  updates of Section 3.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import scipy.linalg

# ---------------------------------------------------------------------------
# Tensor algebra (Section 2.1)
# ---------------------------------------------------------------------------


def mode_product(T: np.ndarray, B: np.ndarray, n: int) -> np.ndarray:
    """Y = T x_n B: Y(i1..j..iN) = sum_{i_n} T(i1..i_n..iN) B(j, i_n) (Section 2.1)."""
    Y = np.tensordot(B, T, axes=([1], [n]))  # (J, remaining modes in order)
    return np.moveaxis(Y, 0, n)


def ttm_qt(T: np.ndarray, Q: np.ndarray, n: int) -> np.ndarray:
    """T x_n Q^T for a factor-shaped Q (I_n x R): mode n shrinks from I_n to R."""
    return mode_product(T, Q.T, n)


def unfold(T: np.ndarray, n: int) -> np.ndarray:
    """Mode-n unfolding, remaining indices flattened in C order (last fastest)."""
    return np.moveaxis(T, n, 0).reshape(T.shape[n], -1)


def unfold_kolda(T: np.ndarray, n: int) -> np.ndarray:
    """Mode-n unfolding in the paper's convention (first remaining index fastest)."""
    return np.moveaxis(T, n, 0).reshape(T.shape[n], -1, order="F")


def kron(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Kronecker product with [A (x) B](K(i-1)+k, L(j-1)+l) = A(i,j) B(k,l) (Section 2.1)."""
    I, J = A.shape
    K, L = B.shape
    out = np.zeros((I * K, J * L))
    for i in range(I):
        for j in range(J):
            out[i * K:(i + 1) * K, j * L:(j + 1) * L] = A[i, j] * B
    return out


def khatri_rao(mats: Sequence[np.ndarray]) -> np.ndarray:
    """Column-wise Kronecker product M_1 (.) M_2 (.) ... (.) M_m (Section 2.1).

    Row index (i_1, ..., i_m) with i_m fastest, i.e. column r is
    kron(m_1r, kron(m_2r, ...)).
    """
    R = mats[0].shape[1]
    out = mats[0].copy()
    for M in mats[1:]:
        out = (out[:, None, :] * M[None, :, :]).reshape(-1, R)
    assert out.shape[1] == R
    return out


def cp_full(lam: np.ndarray, A: Sequence[np.ndarray]) -> np.ndarray:
    """Dense [[lambda; A^(1), ..., A^(N)]] (Section 2.2), summed rank-one term by term."""
    dims = [a.shape[0] for a in A]
    R = A[0].shape[1]
    out = np.zeros(dims)
    for r in range(R):
        term = np.array(lam[r], dtype=np.float64)
        for a in A:
            term = np.multiply.outer(term, a[:, r])
        out += term
    return out


# ---------------------------------------------------------------------------
# Householder QR with positive diagonal (Alg. 2 "calculate QR-decomposition")
# ---------------------------------------------------------------------------


def householder_qr(A: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Compact QR A = Q R of an m x n matrix (m >= n) by Householder reflections.

    Column j: x = W[j:, j]; reflector v = x - a e_1 with a = -sign(x_1)||x||,
    H = I - 2 v v^T / (v^T v).  Q is formed explicitly by applying the
    reflectors in reverse order to the first n columns of I.  Finally the
    signs are fixed so that diag(R) >= 0 (diag(R) > 0 for full column rank).
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if m < n:
        raise ValueError("householder_qr needs m >= n")
    W = A.copy()
    vs: List[Optional[np.ndarray]] = []
    for j in range(n):
        x = W[j:, j]
        nx = np.linalg.norm(x)
        if nx == 0.0:
            vs.append(None)
            continue
        a = -nx if x[0] >= 0 else nx
        v = x.copy()
        v[0] -= a
        v /= np.linalg.norm(v)
        W[j:, j:] -= 2.0 * np.outer(v, v @ W[j:, j:])
        vs.append(v)
    R = np.triu(W[:n, :n])
    Q = np.eye(m, n)
    for j in range(n - 1, -1, -1):
        v = vs[j]
        if v is None:
            continue
        Q[j:, :] -= 2.0 * np.outer(v, v @ Q[j:, :])
    d = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * d[None, :], R * d[:, None]


def solve_upper_transposed(V: np.ndarray, R0: np.ndarray) -> np.ndarray:
    """Solve A^ R0^T = V for A^ (Alg. 2 line 7): back substitution on R0 a_i^T = v_i^T."""
    return scipy.linalg.solve_triangular(R0, V.T, lower=False).T


# ---------------------------------------------------------------------------
# Extrapolation rule (eq. 19 and Section 4.2)
# ---------------------------------------------------------------------------

ALPHA = 0.1
BETA_ACTIVATE_DFIT = 0.03


def beta_band(fit: float) -> float:
    """beta by fit level once extrapolation activates (Section 4.2)."""
    if fit > 0.95:
        return 1.0 / 20000.0
    if fit > 0.90:
        return 1.0 / 2000.0
    if fit > 0.70:
        return 1.0 / 500.0
    return 1.0 / 250.0


class BetaRule:
    """The Section 4.2 controller: feed it each sweep's fit, it returns the beta
    to use in the next sweep (0 until activation, then fixed)."""

    def __init__(self):
        self.fits: List[float] = []
        self.beta = 0.0
        self.activated_after: Optional[int] = None  # 1-based sweep after which beta switched on

    def observe(self, fit: float) -> float:
        self.fits.append(float(fit))
        k = len(self.fits)
        if self.activated_after is None and k >= 2 and abs(self.fits[-1] - self.fits[-2]) < BETA_ACTIVATE_DFIT:
            self.beta = beta_band(self.fits[-1])
            self.activated_after = k
        return self.beta


def extrapolate_q0(Q0: np.ndarray, Q0prev: np.ndarray, beta: float, alpha: float) -> np.ndarray:
    """Customised extrapolation, eq. 19: Q0^ = Q0 + beta (Q0 - alpha Q0prev)."""
    return Q0 + beta * (Q0 - alpha * Q0prev)


# ---------------------------------------------------------------------------
# TTM schedules (Section 3.1, Tables 1-6, Cor. 1)
# ---------------------------------------------------------------------------

TREE_NONE, TREE_STANDARD, TREE_RESTRUCTURED = 0, 1, 2
OP_TTM, OP_UPDATE, OP_FREE = 0, 1, 2


@dataclass
class _Node:
    free: Tuple[int, ...]          # modes still of size I_k
    ver: Dict[int, int]            # contracted mode -> version of Q_k used


# Order-3 restructured tree, sweeps 2 and 3 (repeated with period 2 after
# that): (mode, free set of the source, contraction chain), 0-based modes.
# Sweep 2: A1 from Y(1,3) x3, then Y(2,3) = X x1 -> A2 (x3), A3 (x2).
# Sweep 3: A2 from Y(2,3) x3, then Y(1,3) = X x2 -> A1 (x3), A3 (x1).
# With the standard first sweep this reproduces the item counts of Table 2.
_ORDER3_SWEEPS = [
    [(0, (0, 2), [2]), (1, (0, 1, 2), [0, 2]), (2, (1, 2), [1])],
    [(1, (1, 2), [2]), (0, (0, 1, 2), [1, 2]), (2, (0, 2), [0])],
]

# Order-4 restructured tree, sweeps 2 and 3: (mode, free set of the source,
# contraction chain), 0-based modes.  Reproduces the item counts of Table 5
# together with the standard first sweep.
_ORDER4_SWEEPS = [
    [(2, (2, 3), [3]), (1, (1, 2, 3), [2, 3]), (0, (0, 1, 2, 3), [1, 2, 3]), (3, (0, 3), [0])],
    [(0, (0, 3), [3]), (2, (0, 2, 3), [0, 3]), (1, (0, 1, 2, 3), [2, 0, 3]), (3, (1, 3), [1])],
]


class Schedule:
    """Generates the TTM / update / free operations of each sweep.

    Node 0 is the input tensor X.  Every TTM creates a new node id (counting up
    from 1 over the whole run).  Operations:
      (OP_TTM, dst, src, k)   dst = src x_k Q_k^T with the current Q_k
      (OP_UPDATE, n, leaf)    mode-n update from leaf (all modes but n contracted)
      (OP_FREE, id, 0, 0)     node no longer needed
    """

    def __init__(self, dims: Sequence[int], R: int, tree: int):
        self.dims = [int(d) for d in dims]
        self.N = len(self.dims)
        self.R = int(R)
        self.tree = int(tree)
        self.ver = [0] * self.N
        # per mode: the versions of the other factors its last update saw
        self.seen: Dict[int, Tuple[int, ...]] = {}
        self.nodes: Dict[int, _Node] = {0: _Node(tuple(range(self.N)), {})}
        self.next_id = 1
        self.sweep_index = 0
        self.flops = 0
        self.ops: List[Tuple[int, int, int, int]] = []

    # -- helpers -----------------------------------------------------------
    def node_dims(self, free) -> List[int]:
        return [self.dims[k] if k in free else self.R for k in range(self.N)]

    def ttm_cost(self, free, k) -> int:
        return 2 * self.R * int(np.prod(self.node_dims(free), dtype=np.int64))

    def _valid(self, node: _Node) -> bool:
        return all(self.ver[k] == v for k, v in node.ver.items())

    def _others(self, n: int) -> Tuple[int, ...]:
        return tuple(v for k, v in enumerate(self.ver) if k != n)

    def is_noop(self, n: int) -> bool:
        """An update of mode n now would repeat its last one: no other factor changed since."""
        return self.seen.get(n) == self._others(n)

    def _ttm(self, src: int, k: int) -> int:
        node = self.nodes[src]
        assert k in node.free
        self.flops += self.ttm_cost(node.free, k)
        ver = dict(node.ver)
        ver[k] = self.ver[k]
        dst = self.next_id
        self.next_id += 1
        self.nodes[dst] = _Node(tuple(m for m in node.free if m != k), ver)
        self.ops.append((OP_TTM, dst, src, k))
        return dst

    def _update(self, n: int, leaf: int) -> None:
        assert self.nodes[leaf].free == (n,)
        assert self._valid(self.nodes[leaf])
        self.ops.append((OP_UPDATE, n, leaf, 0))
        self.seen[n] = self._others(n)
        self.ver[n] += 1
        self._free(leaf)
        for i in sorted(self.nodes):
            if i != 0 and n in self.nodes[i].ver:
                self._free(i)

    def _free(self, i: int) -> None:
        del self.nodes[i]
        self.ops.append((OP_FREE, i, 0, 0))

    def _free_all(self) -> None:
        for i in sorted(self.nodes):
            if i != 0:
                self._free(i)

    def _chain(self, src: int, n: int, chain: Sequence[int]) -> None:
        cur = src
        for k in chain:
            cur = self._ttm(cur, k)
        self._update(n, cur)

    # -- the three trees ---------------------------------------------------
    def _no_tree_chain(self, n: int) -> List[int]:
        """Contraction order per mode that reproduces Tables 3 and 6 (no tree)."""
        N = self.N
        if N == 3:
            return [(n - 1) % 3, (n - 2) % 3]
        if n < N // 2:
            return [k for k in range(N - 1, -1, -1) if k != n]
        return [k for k in range(N) if k != n]

    def _standard(self, src: int, m: int, top: bool) -> None:
        """Standard dimension tree on modes 0..m-1 of node src (Tables 1 and 4)."""
        if m == 1:
            self._update(0, src)
            return
        left = self._ttm(src, m - 1)
        self._standard(left, m - 1, False)
        if top and self.N >= 4:
            order = list(range(m - 1))
        else:
            order = list(range(m - 2, -1, -1))
        self._chain(src, m - 1, order)

    def _greedy_step(self, done: set) -> Tuple[int, int, List[int]]:
        best = None
        for n in range(self.N):
            if n in done or self.is_noop(n):
                continue
            for i in sorted(self.nodes):
                node = self.nodes[i]
                if n not in node.free or not self._valid(node):
                    continue
                chain = sorted((k for k in node.free if k != n), key=lambda k: (k not in done, k))
                d = self.node_dims(node.free)
                cost = 0
                for k in chain:
                    cost += 2 * self.R * int(np.prod(d, dtype=np.int64))
                    d[k] = self.R
                key = (cost, n, node.free)
                if best is None or key < best[0]:
                    best = (key, i, n, chain)
        assert best is not None
        return best[1], best[2], best[3]

    def _find(self, free: Tuple[int, ...]) -> int:
        for i in sorted(self.nodes):
            if self.nodes[i].free == tuple(free) and self._valid(self.nodes[i]):
                return i
        raise AssertionError(f"no valid node with free modes {free}")

    def next_sweep(self) -> List[Tuple[int, int, int, int]]:
        """Operations of the next sweep (also appended to self.ops)."""
        start = len(self.ops)
        s = self.sweep_index
        if self.tree == TREE_NONE:
            for n in range(self.N):
                self._chain(0, n, self._no_tree_chain(n))
                self._free_all()
        elif self.tree == TREE_STANDARD or s == 0:
            self._standard(0, self.N, True)
            if self.tree == TREE_STANDARD:
                self._free_all()
        elif self.N == 3:
            for n, free, chain in _ORDER3_SWEEPS[(s - 1) % 2]:
                self._chain(self._find(free), n, chain)
        elif self.N == 4 and s in (1, 2):
            for n, free, chain in _ORDER4_SWEEPS[s - 1]:
                self._chain(self._find(free), n, chain)
        else:
            done: set = set()
            while len(done) < self.N:
                src, n, chain = self._greedy_step(done)
                self._chain(src, n, chain)
                done.add(n)
        self.sweep_index += 1
        return self.ops[start:]


def schedule_ops(dims, R, tree, sweeps) -> List[Tuple[int, int, int, int]]:
    s = Schedule(dims, R, tree)
    for _ in range(sweeps):
        s.next_sweep()
    return s.ops


def schedule_monomial_counts(dims: Sequence[int], R: int, tree: int, sweeps: int):
    """Count the TTMs of the first ``sweeps`` sweeps by cost monomial.

    Key: (free modes of the source, 1-based; power of R).  A TTM on a source
    with free set F costs 2 * prod_{k in F} I_k * R^(N - |F| + 1) (Section 3.4).
    """
    N = len(dims)
    sch = Schedule(dims, R, tree)
    counts: Dict[Tuple[Tuple[int, ...], int], int] = {}
    for _ in range(sweeps):
        sch.next_sweep()
    free_of = {0: tuple(range(N))}
    for op in sch.ops:
        if op[0] == OP_TTM:
            _, dst, src, k = op
            F = free_of[src]
            key = (tuple(m + 1 for m in F), N - len(F) + 1)
            counts[key] = counts.get(key, 0) + 1
            free_of[dst] = tuple(m for m in F if m != k)
    return counts


# ---------------------------------------------------------------------------
# The solver (Alg. 2 / Alg. 3)
# ---------------------------------------------------------------------------


@dataclass
class UpdateRecord:
    sweep: int
    mode: int
    beta: float
    Q0: np.ndarray
    R0: np.ndarray
    V0: np.ndarray
    Vhat: np.ndarray
    A: np.ndarray
    lam: np.ndarray
    Qn: np.ndarray
    Rn: np.ndarray


@dataclass
class Result:
    A: List[np.ndarray]
    lam: np.ndarray
    fits: List[float]
    betas: List[float]
    orders: List[List[int]]
    flops: int
    sweeps: int
    normX2: float
    records: List[UpdateRecord] = field(default_factory=list)


def cp_als_qr(X: np.ndarray, R: int, A0: Sequence[np.ndarray], *, tree: int = TREE_RESTRUCTURED,
              extrapolate: bool = True, alpha: float = ALPHA, beta_fixed: Optional[float] = None,
              max_sweeps: int = 50, tol: float = 0.0, record: bool = False,
              check_leaves: bool = False, beta_schedule: Optional[Sequence[float]] = None,
              on_sweep=None) -> Result:
    """CP-ALS-QR (Alg. 2) with a TTM schedule and optional customised extrapolation (Alg. 3).

    X is promoted to float64 exactly.  A0 are the starting factors (Alg. 2
    "Initialize").  ``beta_fixed`` replaces the Section 4.2 rule with a fixed
    beta from sweep 2 on (ablation); ``beta_schedule[k]`` forces the beta of
    sweep k (0-based) when given.  ``tol`` > 0 stops when |fit_k - fit_{k-1}| < tol.
    ``check_leaves`` asserts every scheduled leaf equals X x_{k != n} Q_k^T.
    ``on_sweep(k, fit)`` is called after every sweep (timing hook; no effect on the result).
    """
    X = np.asarray(X, dtype=np.float64)
    N = X.ndim
    dims = list(X.shape)
    normX2 = float(np.sum(X * X))
    # Initialize: QR of every starting factor.
    Q: List[np.ndarray] = []
    Rf: List[np.ndarray] = []
    for a in A0:
        q, r = householder_qr(np.asarray(a, dtype=np.float64))
        Q.append(q)
        Rf.append(r)
    A = [np.asarray(a, dtype=np.float64).copy() for a in A0]
    lam = np.ones(R)
    Q0prev: List[Optional[np.ndarray]] = [None] * N
    sched = Schedule(dims, R, tree)
    fits: List[float] = []
    betas: List[float] = []
    orders: List[List[int]] = []
    records: List[UpdateRecord] = []
    rule = BetaRule()
    store: Dict[int, np.ndarray] = {0: X}  # cached intermediates, kept across sweeps
    for k in range(max_sweeps):
        if beta_schedule is not None and k < len(beta_schedule):
            beta = float(beta_schedule[k])
        elif not extrapolate:
            beta = 0.0
        elif beta_fixed is not None:
            beta = float(beta_fixed) if k >= 1 else 0.0
        else:
            beta = rule.beta
        betas.append(beta)
        order: List[int] = []
        last = None
        for op in sched.next_sweep():
            kind = op[0]
            if kind == OP_TTM:
                _, dst, src, m = op
                store[dst] = ttm_qt(store[src], Q[m], m)
            elif kind == OP_FREE:
                store.pop(op[1], None)
            else:
                _, n, leaf, _ = op
                Y = store[leaf]
                if check_leaves:
                    direct = X
                    for m in range(N):
                        if m != n:
                            direct = ttm_qt(direct, Q[m], m)
                    assert np.allclose(Y, direct, rtol=1e-12, atol=1e-12 * math.sqrt(normX2))
                # Alg. 3 lines 3-4: Z_n and its QR.
                Z = khatri_rao([Rf[m] for m in range(N) if m != n])
                Q0, R0 = householder_qr(Z)
                # Line 5: customised extrapolation (eq. 19).
                if beta != 0.0 and Q0prev[n] is not None:
                    Q0hat = extrapolate_q0(Q0, Q0prev[n], beta, alpha)
                else:
                    Q0hat = Q0
                # Lines 6-7: V = Y_(n) Q0^ (and V0 = Y_(n) Q0 for the fit).
                Yn = unfold(Y, n)
                V0 = Yn @ Q0
                Vhat = Yn @ Q0hat
                # Line 8: solve A^ R0^T = V.
                Ahat = solve_upper_transposed(Vhat, R0)
                # Line 9: normalise columns.
                lam = np.linalg.norm(Ahat, axis=0)
                A[n] = Ahat / lam[None, :]
                # Line 10: QR of the new factor.
                Q[n], Rf[n] = householder_qr(A[n])
                Q0prev[n] = Q0
                order.append(n)
                last = (V0, Vhat)
                if record:
                    records.append(UpdateRecord(k, n, beta, Q0, R0, V0, Vhat, A[n].copy(), lam.copy(),
                                                Q[n].copy(), Rf[n].copy()))
        orders.append(order)
        V0, Vhat = last
        res2 = normX2 - 2.0 * float(np.sum(V0 * Vhat)) + float(np.sum(Vhat * Vhat))
        fit = 1.0 - math.sqrt(max(res2, 0.0)) / math.sqrt(normX2)
        fits.append(fit)
        # Section 4.2 activation rule.
        rule.observe(fit)
        if on_sweep is not None:
            on_sweep(k, fit)
        if tol > 0 and k >= 1 and abs(fits[-1] - fits[-2]) < tol:
            break
    return Result(A, lam, fits, betas, orders, sched.flops, len(fits), normX2, records)


def fit_explicit(X: np.ndarray, lam: np.ndarray, A: Sequence[np.ndarray]) -> float:
    """Fitness 1 - ||X - K|| / ||X|| with K = [[lambda; A]] formed densely (Section 4.1)."""
    X = np.asarray(X, dtype=np.float64)
    K = cp_full(lam, A)
    return 1.0 - float(np.linalg.norm((X - K).ravel()) / np.linalg.norm(X.ravel()))


# ---------------------------------------------------------------------------
# Cross-checks of one least-squares mode update
# ---------------------------------------------------------------------------


def als_normal_update(X: np.ndarray, A: Sequence[np.ndarray], n: int) -> np.ndarray:
    """CP-ALS mode update (Alg. 1 lines 3-6): A^ Gamma = X_(n) P, Gamma = *_k S_k.

    Returns the unnormalised A^ (C-order KRP matching ``unfold``).
    """
    X = np.asarray(X, dtype=np.float64)
    others = [A[m] for m in range(X.ndim) if m != n]
    Gamma = np.ones((A[0].shape[1], A[0].shape[1]))
    for a in others:
        Gamma = Gamma * (a.T @ a)
    M = unfold(X, n) @ khatri_rao(others)
    return np.linalg.solve(Gamma.T, M.T).T


def qr_update_direct(X: np.ndarray, A: Sequence[np.ndarray], n: int) -> np.ndarray:
    """One CP-ALS-QR mode update from X directly (Alg. 2 lines 3-7), unnormalised A^."""
    X = np.asarray(X, dtype=np.float64)
    N = X.ndim
    Qs, Rs = [], []
    for a in A:
        q, r = householder_qr(a)
        Qs.append(q)
        Rs.append(r)
    Z = khatri_rao([Rs[m] for m in range(N) if m != n])
    Q0, R0 = householder_qr(Z)
    Y = X
    for m in range(N):
        if m != n:
            Y = ttm_qt(Y, Qs[m], m)
    V = unfold(Y, n) @ Q0
    return solve_upper_transposed(V, R0)


# ---------------------------------------------------------------------------
# Small helpers used by the checks
# ---------------------------------------------------------------------------


def subspace_sine(A: np.ndarray, B: np.ndarray) -> float:
    """Largest principal-angle sine between the column spaces of A and B,
    ||(I - Qa Qa^T) Qb||_2, which (unlike sqrt(1 - cos^2)) resolves angles down to rounding."""
    qa, _ = np.linalg.qr(A)
    qb, _ = np.linalg.qr(B)
    return float(np.linalg.norm(qb - qa @ (qa.T @ qb), 2))


def factor_match_score(A_true: Sequence[np.ndarray], A_est: Sequence[np.ndarray], lam_true=None, lam_est=None) -> float:
    """Mean over components of prod_n |cos(a_true_r, a_est_pi(r))| under the best greedy matching."""
    R = A_true[0].shape[1]
    C = np.ones((R, R))
    for at, ae in zip(A_true, A_est):
        at = at / np.linalg.norm(at, axis=0)
        ae = ae / np.linalg.norm(ae, axis=0)
        C = C * np.abs(at.T @ ae)
    used = set()
    total = 0.0
    for r in np.argsort(-C.max(axis=1)):
        best = max((c for c in range(R) if c not in used), key=lambda c: C[r, c])
        used.add(best)
        total += C[r, best]
    return total / R
