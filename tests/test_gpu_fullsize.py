"""Parity at the benchmark workloads' full sizes: the 400^3 rank-32 tensor (FP64 path and
split-precision path, the configuration bench.py times), and one sweep of the 128^4 rank-24
and 48^5 rank-16 workloads, against the FP64 oracle run on the same tensors."""
import numpy as np
import pytest

from oracle import cpqr_oracle as o
from paper_2503_18759_gb300 import binding as b
from paper_2503_18759_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2503_18759_gb300 import build
    build.build()
    b.lib()


@pytest.fixture(scope="module")
def cube400():
    return inputs.workload("cube400_r32_c09", seed=0)


def _gpu(prob, prec, sweeps, extrap=b.EXTRAP_PAPER):
    X = torch.from_numpy(prob.X).to(DEV)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=prec, extrap=extrap)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
        fits = d.sweep(sweeps)
        A, lam, Q, _ = d.factors()
    return fits, A, lam, Q


def test_cube400_fp64_path_three_sweeps(cube400):
    """FP64 path on the full 400^3 tensor: fits and factor subspaces within 1e-10 of the oracle
    over the standard first sweep and two restructured sweeps."""
    fits, A, lam, Q = _gpu(cube400, b.PREC_FP64, 3)
    ref = o.cp_als_qr(cube400.X, cube400.R, cube400.A0, tree=o.TREE_RESTRUCTURED, max_sweeps=3)
    assert np.max(np.abs(fits - np.array(ref.fits))) <= 1e-10
    for n in range(3):
        assert o.subspace_sine(A[n], ref.A[n]) <= 1e-10
        assert np.allclose(Q[n].T @ Q[n], np.eye(32), atol=1e-13)


def split_fit_tol(fit_ref):
    """Per-sweep fit tolerance of the split path: the bf16 hi + lo operands carry ~2^-17 relative
    error, so ||V0||^2 (and <V0, V^>) carry ~2^-16 of ||X||^2, which moves
    1 - sqrt(||X||^2 - ||V0||^2)/||X|| by ~2^-16 / (2 (1 - fit)); a factor 4 of margin."""
    return 2.0 ** -15 / (1.0 - np.asarray(fit_ref))


def test_cube400_split_precision_three_sweeps(cube400):
    """Split-precision path (tcgen05 full-tensor TTMs, FP32 deeper TTMs, FP64 QRs) on the full
    400^3 tensor against the FP64 oracle: per-sweep fits within split_fit_tol; factor subspaces
    within 2e-3 (2^-16 operand error times the conditioning of congruence-0.9 factors)."""
    fits, A, lam, Q = _gpu(cube400, b.PREC_SPLIT_BF16, 3)
    ref = o.cp_als_qr(cube400.X, cube400.R, cube400.A0, tree=o.TREE_RESTRUCTURED, max_sweeps=3)
    rf = np.array(ref.fits)
    assert np.all(np.abs(fits - rf) <= split_fit_tol(rf)), (fits, rf)
    for n in range(3):
        assert o.subspace_sine(A[n], ref.A[n]) <= 2e-3


@pytest.mark.parametrize("name", ["hyper128_r24_c08", "order5_48_r16"])
def test_order4_and_order5_workloads_first_sweep(name):
    """One restructured-tree sweep (the standard first sweep) of the 128^4 and 48^5 workloads.
    FP64 path: fit and factor subspaces within 1e-9 of the oracle.  Split path: fit within
    split_fit_tol, factor subspaces within 10x the oracle's own change when X is perturbed by a
    random 2^-16 relative amount (the size of the split operands' error): after one sweep from a
    random start the factors can be ill-conditioned, so the bound is measured, not assumed."""
    prob = inputs.workload(name, seed=0)
    ref = o.cp_als_qr(prob.X, prob.R, prob.A0, tree=o.TREE_RESTRUCTURED, extrapolate=False, max_sweeps=1)
    f64, A64, _, _ = _gpu(prob, b.PREC_FP64, 1, extrap=b.EXTRAP_NONE)
    assert abs(f64[0] - ref.fits[0]) <= 1e-9
    for n in range(len(prob.dims)):
        assert o.subspace_sine(A64[n], ref.A[n]) <= 1e-9
    g = np.random.default_rng(1)
    Xp = prob.X.astype(np.float64)
    Xp *= 1.0 + 2.0 ** -16 * g.standard_normal(Xp.shape)
    ref_p = o.cp_als_qr(Xp, prob.R, prob.A0, tree=o.TREE_RESTRUCTURED, extrapolate=False, max_sweeps=1)
    del Xp
    fits, A, lam, Q = _gpu(prob, b.PREC_SPLIT_BF16, 1, extrap=b.EXTRAP_NONE)
    assert abs(fits[0] - ref.fits[0]) <= split_fit_tol(ref.fits[0])
    for n in range(len(prob.dims)):
        sens = o.subspace_sine(ref_p.A[n], ref.A[n])
        assert o.subspace_sine(A[n], ref.A[n]) <= 10 * max(sens, 1e-6), (n, sens)
