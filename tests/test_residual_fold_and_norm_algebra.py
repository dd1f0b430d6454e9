"""Host restatements of two pieces of kernel arithmetic (no GPU):

* the explicit residual's folded view (csrc/residual_tc.cu): X in C order viewed as rows over the
  leading modes and columns over the trailing nt modes, nt grown from 1 while the columns are
  fewer than 128; the model block is W B^T with W the Khatri-Rao weights of the row modes (lambda
  in the first factor) and B those of the column modes, each row and column index decomposed with
  its last mode fastest.  ||X - W B^T||^2 over the view equals the dense residual of the CP model
  (the fit of Section 4.1 without the reduced form).
* the float-float sum of squares of an FP32 tensor (csrc/ttm.cu::norm2_f32_kernel): each square
  kept exactly as (p, e) with p = fl(x x), the two summed over runs of 16 with a two-sum on the
  high part, each run then added in FP64; emulated with IEEE float32 arithmetic in numpy, its error
  against the exact sum stays within the bound the kernel's comment states."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import cpqr_oracle as o

FOLD = 128  # the residual's column threshold


def _fold(dims):
    """(nt, columns): trailing modes taken into the columns while they are fewer than FOLD."""
    N = len(dims)
    nt, ic = 1, dims[-1]
    while ic < FOLD and nt < N - 1:
        ic *= dims[N - 1 - nt]
        nt += 1
    return nt, ic


def _digits(idx, ds):
    """Mixed-radix digits of idx over the dims ds, the last one fastest."""
    out = []
    for d in reversed(ds):
        out.append(idx % d)
        idx //= d
    return list(reversed(out))


@pytest.mark.parametrize("dims,R", [([37, 29, 36], 6), ([20, 30, 260], 8), ([6, 5, 7, 4, 8], 4), ([3, 4, 8], 3),
                                    ([9, 7, 5, 6], 5), ([48, 48, 48], 4)])
def test_folded_view_residual_equals_dense_residual(dims, R):
    g = np.random.default_rng(sum(dims) + R)
    A = [g.standard_normal((d, R)) for d in dims]
    lam = g.uniform(0.5, 2.0, R)
    X = g.standard_normal(dims)
    nt, ic = _fold(dims)
    row_dims, col_dims = dims[:len(dims) - nt], dims[len(dims) - nt:]
    rows = int(np.prod(row_dims))
    assert rows * ic == X.size
    # weights of the rows (lambda in the first factor) and of the columns, index by index
    W = np.ones((rows, R))
    for r in range(rows):
        for n, i in enumerate(_digits(r, row_dims)):
            W[r] *= A[n][i] * (lam if n == 0 else 1.0)
    B = np.ones((ic, R))
    off = len(row_dims)
    for c in range(ic):
        for n, i in enumerate(_digits(c, col_dims)):
            B[c] *= A[off + n][i]
    K = W @ B.T
    res_view = float(np.sum((X.reshape(rows, ic) - K) ** 2))
    dense = np.einsum("r,ir,jr->ij", lam, A[0], o.khatri_rao(A[1:])).reshape(dims)
    res_dense = float(np.sum((X - dense) ** 2))
    assert abs(res_view - res_dense) <= 1e-10 * res_dense
    # the fold rule: at least FOLD columns unless every mode but the first is folded, and no more
    # modes than needed
    assert ic >= FOLD or nt == len(dims) - 1
    if nt > 1:
        assert int(np.prod(dims[len(dims) - nt + 1:])) < FOLD


def _ff_norm(x32: np.ndarray) -> float:
    """The kernel's per-thread arithmetic over one sequence of FP32 values, in IEEE float32."""
    f32 = np.float32
    acc = 0.0
    hi, lo, run = f32(0), f32(0), 0
    for x in x32:
        x = f32(x)
        ax = abs(x)
        if not (ax < f32(1e18) and (ax >= f32(1e-15) or x == 0)):
            acc += float(x) * float(x)
            continue
        p = f32(x * x)
        e = f32(float(x) * float(x) - float(p))  # fma(x, x, -p): exact, x * x has <= 48 bits
        s = f32(hi + p)
        bb = f32(s - hi)
        t = f32(f32(hi - f32(s - bb)) + f32(p - bb))
        hi = s
        lo = f32(lo + f32(t + e))
        run += 1
        if run == 16:
            acc += float(hi) + float(lo)
            hi, lo, run = f32(0), f32(0), 0
    return acc + float(hi) + float(lo)


@pytest.mark.parametrize("scale,n", [(1.0, 1000), (1e3, 777), (3e-7, 500), (1e17, 64)])
def test_float_float_sum_of_squares_within_its_bound(scale, n):
    g = np.random.default_rng(n)
    x = (g.standard_normal(n) * scale).astype(np.float32)
    exact = sum(Fraction(float(v)) ** 2 for v in x)
    got = _ff_norm(x)
    err = abs(Fraction(got) - exact) / exact
    runs = math.ceil(n / 16)
    # float-float error of a run: ~16 * 2^-48 of it; the FP64 additions of the runs: runs * 2^-53
    assert err <= 16 * 2.0 ** -48 + runs * 2.0 ** -53, float(err)


def test_out_of_range_values_take_the_fp64_squares():
    x = np.array([1e19, 1e-20, 0.0, 2.0, -3e18], dtype=np.float32)
    exact = sum(Fraction(float(v)) ** 2 for v in x)
    got = _ff_norm(x)
    assert abs(Fraction(got) - exact) / exact <= 1e-15
    assert math.isinf(_ff_norm(np.array([np.inf, 1.0], dtype=np.float32)))
    assert math.isnan(_ff_norm(np.array([np.nan, 1.0], dtype=np.float32)))
