"""Seeded synthetic inputs for CP-ALS-QR (tensors, true factors, initial factors).

This module only *draws* inputs; it contains none of the decomposition's own
arithmetic (no TTM, no QR of the method, no least-squares solve).  Both the
CUDA path and the CPU oracle consume what it returns.

Construction follows the synthetic-tensor recipe of Section 4.2 (subsection
"Synthetic tensors"): per mode an R x R congruence matrix K with unit diagonal
and off-diagonal c, its upper Cholesky factor C (K = C^T C), a standard-normal
I x R matrix orthonormalised column-wise to Q, and the factor B = Q C, so the
columns of B have unit norm and pairwise cosine exactly c.  Homoscedastic
noise is added as X' = X + eta * (||X|| / ||N||) * N with N standard normal;
the paper's percentage parameter l1 maps to eta = 1 / sqrt(100 / l1 - 1).

Every tensor is dense and stored in C order (last index fastest).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

# Stream identifiers: one independent PCG64 stream per purpose, so that
# changing e.g. the noise level never changes the factors.
_STREAM_FACTORS = 1
_STREAM_NOISE = 2
_STREAM_INIT = 3


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


def eta_from_l1(l1: float) -> float:
    """Relative noise norm for the paper's homoscedastic level l1 (percent)."""
    if l1 <= 0:
        return 0.0
    return 1.0 / math.sqrt(100.0 / l1 - 1.0)


def gaussian_factors(dims: Sequence[int], R: int, seed: int, stream: int = _STREAM_FACTORS) -> List[np.ndarray]:
    """I_n x R factor matrices with i.i.d. N(0,1) entries (float64)."""
    g = _rng(seed, stream)
    return [g.standard_normal((int(I), R)) for I in dims]


def collinear_factors(dims: Sequence[int], R: int, c, seed: int) -> List[np.ndarray]:
    """Factors B = Q C with unit columns of pairwise cosine c (Section 4.2).

    ``c`` is a scalar or one value per mode.
    """
    g = _rng(seed, _STREAM_FACTORS)
    cs = list(c) if isinstance(c, (list, tuple, np.ndarray)) else [float(c)] * len(dims)
    out = []
    for I, cn in zip(dims, cs):
        K = (1.0 - cn) * np.eye(R) + cn * np.ones((R, R))
        C = np.linalg.cholesky(K).T  # upper, K = C^T C
        M = g.standard_normal((int(I), R))
        Q, _ = np.linalg.qr(M)  # thin QR: orthonormal columns
        out.append(Q @ C)
    return out


def cp_dense(factors: Sequence[np.ndarray], weights: Optional[np.ndarray] = None) -> np.ndarray:
    """Dense C-order tensor sum_r w_r b_r^(1) o ... o b_r^(N) (float64)."""
    R = factors[0].shape[1]
    w = np.ones(R) if weights is None else np.asarray(weights, dtype=np.float64)
    rows = factors[0]
    for B in factors[1:-1]:
        rows = (rows[:, None, :] * B[None, :, :]).reshape(-1, R)
    X = rows @ (w[:, None] * factors[-1].T)
    return X.reshape([f.shape[0] for f in factors])


def add_noise(X: np.ndarray, eta: float, seed: int) -> np.ndarray:
    """X + eta * ||X||/||N|| * N, N i.i.d. N(0,1) (homoscedastic, Section 4.2)."""
    if eta <= 0:
        return X.copy()
    g = _rng(seed, _STREAM_NOISE)
    Nz = g.standard_normal(X.shape)
    return X + (eta * np.linalg.norm(X.ravel()) / np.linalg.norm(Nz.ravel())) * Nz


def init_factors(dims: Sequence[int], R: int, seed: int) -> List[np.ndarray]:
    """Random N(0,1) starting factors A^(n) (the 'Initialize' step of Alg. 2/3)."""
    return gaussian_factors(dims, R, seed, stream=_STREAM_INIT)


@dataclass
class Problem:
    """One seeded CP problem: tensor, its true factors and a starting point."""
    name: str
    dims: List[int]
    R: int
    X: np.ndarray                      # C-order, float32 or float64
    A0: List[np.ndarray]               # starting factors, float64, I_n x R
    true_factors: List[np.ndarray]
    eta: float
    seed: int
    meta: dict = field(default_factory=dict)


def make_problem(name: str, dims: Sequence[int], R: int, *, seed: int, c=None, eta: float = 0.0,
                 dtype=np.float32, true_rank: Optional[int] = None) -> Problem:
    """Build a seeded problem.

    c=None draws i.i.d. N(0,1) true factors (config of the 60^3 case); a number
    (or per-mode list) uses the collinear construction of Section 4.2.
    """
    dims = [int(d) for d in dims]
    Rt = R if true_rank is None else int(true_rank)
    if c is None:
        B = gaussian_factors(dims, Rt, seed)
    else:
        B = collinear_factors(dims, Rt, c, seed)
    X = add_noise(cp_dense(B), eta, seed)
    X = np.ascontiguousarray(X.astype(dtype))
    A0 = init_factors(dims, R, seed)
    return Problem(name, dims, R, X, A0, B, eta, seed, {"c": c, "dtype": np.dtype(dtype).name})


# The workloads.  Sizes and statistics follow the configurations the method is
# evaluated on; the 1e-3 / 1e-4 noise values are relative Frobenius norms.
WORKLOADS = {
    "cube60_r5_f64": dict(dims=[60, 60, 60], R=5, c=None, eta=1e-4, dtype=np.float64),
    "cube400_r32_c09": dict(dims=[400, 400, 400], R=32, c=0.9, eta=1e-3, dtype=np.float32),
    "hyper128_r24_c08": dict(dims=[128] * 4, R=24, c=0.8, eta=1e-3, dtype=np.float32),
    "order5_48_r16": dict(dims=[48] * 5, R=16, c=None, eta=1e-4, dtype=np.float32),
}


def workload(name: str, seed: int = 0, **overrides) -> Problem:
    cfg = dict(WORKLOADS[name])
    cfg.update(overrides)
    return make_problem(name, cfg.pop("dims"), cfg.pop("R"), seed=seed, **cfg)


def make_problem_device(name: str, dims: Sequence[int], R: int, *, seed: int, c=None, eta: float = 0.0,
                        device: str = "cuda"):
    """Same recipe as make_problem, with the dense tensor and the noise formed on the GPU by
    torch (seeded torch generator) for large training sets; X is a float32 device tensor.
    Factors and starting factors are drawn with numpy exactly as in make_problem."""
    import torch

    dims = [int(d) for d in dims]
    B = gaussian_factors(dims, R, seed) if c is None else collinear_factors(dims, R, c, seed)
    Bt = [torch.from_numpy(b).to(device) for b in B]
    rows = Bt[0]
    for Bn in Bt[1:-1]:
        rows = (rows[:, None, :] * Bn[None, :, :]).reshape(-1, R)
    X = (rows @ Bt[-1].T).reshape(dims)
    if eta > 0:
        gen = torch.Generator(device=device)
        gen.manual_seed(int(seed) * 7919 + _STREAM_NOISE)
        Nz = torch.randn(dims, generator=gen, device=device, dtype=torch.float64)
        X = X + (eta * torch.linalg.vector_norm(X) / torch.linalg.vector_norm(Nz)) * Nz
    X = X.to(torch.float32).contiguous()
    return Problem(name, dims, R, X, init_factors(dims, R, seed), B, eta, seed, {"c": c, "dtype": "float32"})
