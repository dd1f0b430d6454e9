"""The wide-rank path (32 < R <= 192, the high-rank regime of Table 7) against the FP64 oracle:
its Cholesky QRs (factor and Khatri-Rao) against the oracle's Householder QR, the solver on both
paths, and the explicit residual."""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("M,R,kappa", [(200, 40, 1.0), (400, 64, 1.0), (1000, 150, 1.0), (192, 192, 1.0),
                                       (500, 100, 1e7)])
def test_wide_factor_qr_matches_householder(M, R, kappa):
    """Unit columns (the factors of a sweep are normalised); kappa = 1e7 makes the first Cholesky
    pass leave |Q^T Q - I| ~ 1e-2, so the second pass runs.  Q R reproduces A to rounding, Q is
    orthonormal, and both equal the oracle's Householder factors (positive diagonal) to
    kappa-scaled rounding."""
    g = np.random.default_rng(M + R)
    A = g.standard_normal((M, R))
    if kappa > 1:
        U, _ = np.linalg.qr(A)
        V, _ = np.linalg.qr(g.standard_normal((R, R)))
        A = U @ np.diag(np.logspace(0, -np.log10(kappa), R)) @ V.T
    A /= np.linalg.norm(A, axis=0)
    Qr, Rr = o.householder_qr(A)
    Q = torch.empty((M, R), dtype=torch.float64, device=DEV)
    Rm = torch.empty((R, R), dtype=torch.float64, device=DEV)
    Ad = _dev(A)
    b.cpqr_house_qr(Ad.data_ptr(), M, R, Q.data_ptr(), Rm.data_ptr())
    torch.cuda.synchronize()
    Qg, Rg = Q.cpu().numpy(), Rm.cpu().numpy()
    assert np.abs(Qg.T @ Qg - np.eye(R)).max() < 1e-13
    assert np.abs(Qg @ Rg - A).max() < 1e-13
    assert np.all(np.diag(Rg) > 0) and np.abs(np.tril(Rg, -1)).max() == 0.0
    assert np.abs(Rg - Rr).max() <= 1e-12 * max(kappa, 1.0)
    assert np.abs(Qg - Qr).max() <= 1e-11 * max(kappa, 1.0)


@pytest.mark.parametrize("m,R", [(2, 40), (2, 64), (3, 36), (2, 150), (1, 48)])
def test_wide_khatri_rao_qr_matches_householder(m, R):
    g = np.random.default_rng(10 * m + R)
    tri = []
    for _ in range(m):
        B = g.standard_normal((R + 7, R))
        B /= np.linalg.norm(B, axis=0)
        tri.append(o.householder_qr(B)[1])
    Z = o.khatri_rao(tri)
    Q0r, R0r = o.householder_qr(Z)
    Q0 = torch.empty(Z.shape, dtype=torch.float64, device=DEV)
    R0 = torch.empty((R, R), dtype=torch.float64, device=DEV)
    Rd = _dev(np.stack(tri))
    b.cpqr_krp_qr(Rd.data_ptr(), m, R, Q0.data_ptr(), R0.data_ptr())
    torch.cuda.synchronize()
    Qg, Rg = Q0.cpu().numpy(), R0.cpu().numpy()
    assert np.abs(Qg.T @ Qg - np.eye(R)).max() < 1e-13
    assert np.abs(Qg @ Rg - Z).max() < 1e-13 * np.abs(Z).max()
    assert np.allclose(Rg, R0r, atol=1e-12 * np.abs(R0r).max())
    assert np.allclose(Qg, Q0r, atol=1e-11)


WIDE = [("r64_order3", [70, 66, 68], 64, b.EXTRAP_FIXED, 0.01, 4),
        ("r150_order3", [160, 154, 156], 150, b.EXTRAP_FIXED, 0.01, 3),
        ("r36_order4", [40, 38, 39, 37], 36, b.EXTRAP_NONE, 0.0, 3)]


@pytest.mark.parametrize("name,dims,R,extrap,beta,sweeps", WIDE, ids=[w[0] for w in WIDE])
def test_wide_fp64_solver_matches_oracle(name, dims, R, extrap, beta, sweeps):
    """The restructured tree at ranks 36 .. 150 on the FP64 path: fits and factor subspaces within
    1e-10 of the oracle (Householder QRs throughout), lambda to 1e-8."""
    prob = inputs.make_problem(name, dims, R, seed=6, c=0.3, eta=1e-3, dtype=np.float64)
    X = _dev(prob.X)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_FP64, extrap=extrap, beta_fixed=beta)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), True, prob.A0, opts) as d:
        fits = d.sweep(sweeps)
        A, lam, Q, Rn = d.factors()
    kw = dict(extrapolate=False) if extrap == b.EXTRAP_NONE else dict(extrapolate=True, beta_fixed=beta)
    ref = o.cp_als_qr(prob.X, prob.R, prob.A0, tree=o.TREE_RESTRUCTURED, max_sweeps=sweeps, **kw)
    assert np.max(np.abs(fits - np.array(ref.fits))) <= 1e-10, (fits, ref.fits)
    for n in range(len(dims)):
        assert o.subspace_sine(A[n], ref.A[n]) <= 1e-10
        assert np.abs(Q[n].T @ Q[n] - np.eye(R)).max() < 1e-13
        assert np.all(np.diag(Rn[n]) > 0)
    assert np.allclose(lam, ref.lam, rtol=1e-8)


def _sensitivity(prob, sweeps, **kw):
    """The oracle's own factor change when X is perturbed by a random 2^-16 relative amount (the
    split operands' error): the subspace bound of the split path is 10x this, measured."""
    g = np.random.default_rng(1)
    Xp = prob.X.astype(np.float64) * (1.0 + 2.0 ** -16 * g.standard_normal(prob.X.shape))
    ref = o.cp_als_qr(prob.X, prob.R, prob.A0, tree=o.TREE_RESTRUCTURED, max_sweeps=sweeps, **kw)
    ref_p = o.cp_als_qr(Xp, prob.R, prob.A0, tree=o.TREE_RESTRUCTURED, max_sweeps=sweeps, **kw)
    return ref, [o.subspace_sine(ref_p.A[n], ref.A[n]) for n in range(len(prob.dims))]


def test_wide_split_precision_solver_tracks_oracle():
    """The split path at R = 64 (FP32 tensor; its last side, 68, is not a multiple of 8, so the
    TTMs over the tensor take the tensor cores through the padded split copy, the deeper ones the
    CUDA cores; FP64 QRs, explicit residual fit): per-sweep fits within
    1e-4 of the oracle, factor subspaces within 10x the oracle's own change under a 2^-16 relative
    perturbation of X (R = 64 of 68 columns makes the factors' subspaces sensitive)."""
    prob = inputs.make_problem("wide_split", [72, 70, 68], 64, seed=7, c=0.3, eta=1e-2, dtype=np.float32)
    X = _dev(prob.X)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_SPLIT_BF16, extrap=b.EXTRAP_FIXED, beta_fixed=0.01)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
        fits = d.sweep(5)
        A, lam, _, _ = d.factors()
        fx = d.fit_exact()
    ref, sens = _sensitivity(prob, 5, extrapolate=True, beta_fixed=0.01)
    assert np.max(np.abs(fits - np.array(ref.fits))) <= 1e-4, (fits, ref.fits)
    for n in range(3):
        assert o.subspace_sine(A[n], ref.A[n]) <= 10 * max(sens[n], 1e-6), (n, sens[n])
    assert abs(fx - o.fit_explicit(prob.X, lam, A)) <= 1e-7


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_wide_fit_exact_matches_dense_residual(dtype):
    prob = inputs.make_problem("wide_fx", [50, 52, 60], 48, seed=12, c=0.4, eta=3e-3, dtype=dtype)
    X = _dev(prob.X)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_FP64, extrap=b.EXTRAP_NONE)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), dtype == np.float64, prob.A0, opts) as d:
        fits = d.sweep(4)
        A, lam, _, _ = d.factors()
        fx = d.fit_exact()
    ref = o.fit_explicit(prob.X, lam, A)
    assert abs(fx - ref) <= 1e-8
    assert abs(fits[-1] - ref) <= 1e-8


def test_wide_split_solver_on_the_tensor_cores_tracks_oracle():
    """The split path at R = 48 with every TTM on the wide tensor-core kernel (sides multiples of 8):
    per-sweep fits within 1e-4 of the oracle, factor subspaces within 10x the oracle's sensitivity."""
    prob = inputs.make_problem("wide_tc", [64, 56, 72], 48, seed=8, c=0.3, eta=1e-2, dtype=np.float32)
    X = _dev(prob.X)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_SPLIT_BF16, extrap=b.EXTRAP_NONE)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
        fits = d.sweep(5)
        A, lam, _, _ = d.factors()
    ref, sens = _sensitivity(prob, 5, extrapolate=False)
    assert np.max(np.abs(fits - np.array(ref.fits))) <= 1e-4, (fits, ref.fits)
    for n in range(3):
        assert o.subspace_sine(A[n], ref.A[n]) <= 10 * max(sens[n], 1e-6), (n, sens[n])


def test_wide_lagged_fit_equals_sweep_by_sweep_fit():
    """On the wide path the split solver's explicit residual (CUDA cores) is read one sweep late
    inside a multi-sweep call too, beside the next sweep; the fits, betas and factors equal those of
    sweep-by-sweep reads, up to the order of the residual's block partials."""
    prob = inputs.make_problem("wide_lag", [64, 56, 72], 48, seed=8, c=0.3, eta=1e-2, dtype=np.float32)
    X = _dev(prob.X)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_SPLIT_BF16, extrap=b.EXTRAP_FIXED, beta_fixed=0.01)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
        f_many = d.sweep(10)
        A1, lam1, _, _ = d.factors()
        lagged = d.stats().lagged_fits
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
        f_one = np.array([d.sweep(1)[0] for _ in range(10)])
        A2, lam2, _, _ = d.factors()
    assert lagged >= 1
    assert np.allclose(f_many, f_one, rtol=0, atol=1e-12), (f_many - f_one)
    for a1, a2 in zip(A1, A2):
        assert np.array_equal(a1, a2)
    assert np.array_equal(lam1, lam2)
