"""GPU parity: every step of the CUDA path against the FP64 CPU oracle on the
same seeded inputs, through the C ABI."""
import math

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
    assert torch.cuda.is_available()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _rel(a, ref):
    return float(np.max(np.abs(a - ref)) / max(np.max(np.abs(ref)), 1e-300))


# ragged tails; S == 1 with K % 4 == 0 and S % 4 == 0 reach the register-tiled FP32 kernel,
# the other shapes the generic one
TTM_SHAPES = [((37, 53, 29), 5), ((64, 65, 66), 32), ((9, 10, 11, 12), 7), ((3, 200, 2), 2), ((130, 7, 1, 5), 1),
              ((5, 6, 7, 8, 9), 4), ((128, 128, 3), 24), ((300, 32, 400), 32), ((32, 400, 132), 24),
              ((9, 8, 12, 20), 16)]


@pytest.mark.parametrize("dims,R", TTM_SHAPES)
def test_ttm_fp64_every_mode(dims, R):
    g = np.random.default_rng(sum(dims) + R)
    T = g.standard_normal(dims)
    for k in range(len(dims)):
        if dims[k] < 1:
            continue
        Q = g.standard_normal((dims[k], R))
        ref = o.ttm_qt(T, Q, k)
        out = torch.empty(ref.shape, dtype=torch.float64, device=DEV)
        Td, Qd = _dev(T), _dev(Q)  # keep the device copies alive across the call
        b.cpqr_ttm(Td.data_ptr(), dims, k, Qd.data_ptr(), R, out.data_ptr(), b.TTM_F64)
        torch.cuda.synchronize()
        assert _rel(out.cpu().numpy(), ref) < 1e-13, (dims, k)


@pytest.mark.parametrize("dims,R", TTM_SHAPES)
def test_ttm_fp32_every_mode(dims, R):
    g = np.random.default_rng(sum(dims) + R + 1)
    T = g.standard_normal(dims).astype(np.float32)
    for k in range(len(dims)):
        Q = g.standard_normal((dims[k], R)).astype(np.float32)
        ref = o.ttm_qt(T.astype(np.float64), Q.astype(np.float64), k)
        Td, Qd = _dev(T), _dev(Q)
        out = torch.empty(ref.shape, dtype=torch.float32, device=DEV)
        b.cpqr_ttm(Td.data_ptr(), dims, k, Qd.data_ptr(), R, out.data_ptr(), b.TTM_F32)
        out64 = torch.empty(ref.shape, dtype=torch.float64, device=DEV)
        Q64 = _dev(Q.astype(np.float64))
        b.cpqr_ttm(Td.data_ptr(), dims, k, Q64.data_ptr(), R, out64.data_ptr(), b.TTM_F32_IN_F64)
        torch.cuda.synchronize()
        # FP32 accumulation over K terms: |err| <= K * 2^-24 * sum|t q|, checked loosely against max|ref|
        K = dims[k]
        assert _rel(out.cpu().numpy(), ref) < 4 * math.sqrt(K) * 2 ** -24 * 8
        assert _rel(out64.cpu().numpy(), ref) < 1e-13


@pytest.mark.parametrize("M,R", [(400, 32), (60, 5), (33, 32), (1000, 17), (5, 5), (128, 24), (2049, 32)])
def test_house_qr(M, R):
    g = np.random.default_rng(M * 7 + R)
    A = g.standard_normal((M, R))
    Qr, Rr = o.householder_qr(A)
    Q = torch.empty((M, R), dtype=torch.float64, device=DEV)
    Rm = torch.empty((R, R), dtype=torch.float64, device=DEV)
    Ad = _dev(A)
    b.cpqr_house_qr(Ad.data_ptr(), M, R, Q.data_ptr(), Rm.data_ptr())
    torch.cuda.synchronize()
    assert np.allclose(Rm.cpu().numpy(), Rr, atol=1e-12 * np.linalg.norm(A))
    assert np.allclose(Q.cpu().numpy(), Qr, atol=1e-12)


@pytest.mark.parametrize("m,R", [(2, 5), (2, 32), (3, 24), (4, 16), (2, 1), (3, 7), (4, 5), (3, 32), (4, 17)])
def test_krp_qr(m, R):
    g = np.random.default_rng(m * 100 + R)
    Rs = [o.householder_qr(g.standard_normal((R + 4, R)))[1] for _ in range(m)]
    Z = o.khatri_rao(Rs)
    Q0r, R0r = o.householder_qr(Z)
    Q0 = torch.empty(Z.shape, dtype=torch.float64, device=DEV)
    R0 = torch.empty((R, R), dtype=torch.float64, device=DEV)
    Rd = _dev(np.stack(Rs))
    b.cpqr_krp_qr(Rd.data_ptr(), m, R, Q0.data_ptr(), R0.data_ptr())
    torch.cuda.synchronize()
    assert np.allclose(R0.cpu().numpy(), R0r, atol=1e-12 * np.abs(R0r).max())
    assert np.allclose(Q0.cpu().numpy(), Q0r, atol=1e-11)


def _run_gpu(prob, tree, extrap, beta_fixed, sweeps, prec=b.PREC_FP64, route=b.QR_GRAM):
    x64 = prob.X.dtype == np.float64
    X = _dev(prob.X)
    opts = b.make_options(tree=tree, prec=prec, extrap=extrap, beta_fixed=beta_fixed, qr_route=route)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), x64, prob.A0, opts) as d:
        fits = d.sweep(sweeps)
        A, lam, Q, Rn = d.factors()
        st = d.stats()
    return fits, A, lam, Q, Rn, st


def _run_oracle(prob, tree, extrap, beta_fixed, sweeps):
    kw = dict(tree=tree, max_sweeps=sweeps)
    if extrap == b.EXTRAP_NONE:
        kw["extrapolate"] = False
    elif extrap == b.EXTRAP_FIXED:
        kw.update(extrapolate=True, beta_fixed=beta_fixed)
    else:
        kw["extrapolate"] = True
    return o.cp_als_qr(prob.X, prob.R, prob.A0, **kw)


CASES = [
    ("cube60_std", dict(dims=[60, 60, 60], R=5, c=None, eta=1e-4, dtype=np.float64), b.TREE_STANDARD, b.EXTRAP_NONE, 0.0, 12),
    ("order3_rest_fixed", dict(dims=[23, 19, 17], R=6, c=0.6, eta=1e-2, dtype=np.float64), b.TREE_RESTRUCTURED, b.EXTRAP_FIXED, 0.02, 8),
    ("order3_rest_paper", dict(dims=[30, 31, 29], R=8, c=0.9, eta=1e-3, dtype=np.float32), b.TREE_RESTRUCTURED, b.EXTRAP_PAPER, 0.0, 10),
    ("order4_rest", dict(dims=[11, 9, 10, 12], R=4, c=0.5, eta=1e-3, dtype=np.float64), b.TREE_RESTRUCTURED, b.EXTRAP_FIXED, 0.01, 7),
    ("order4_std", dict(dims=[11, 9, 10, 12], R=4, c=0.5, eta=1e-3, dtype=np.float32), b.TREE_STANDARD, b.EXTRAP_NONE, 0.0, 5),
    ("order5_rest", dict(dims=[6, 7, 5, 6, 7], R=3, c=None, eta=1e-3, dtype=np.float64), b.TREE_RESTRUCTURED, b.EXTRAP_FIXED, 0.01, 6),
    ("order3_none", dict(dims=[15, 16, 17], R=5, c=0.3, eta=1e-3, dtype=np.float64), b.TREE_NONE, b.EXTRAP_NONE, 0.0, 5),
    ("order3_r32", dict(dims=[40, 36, 33], R=32, c=0.5, eta=1e-3, dtype=np.float64), b.TREE_RESTRUCTURED, b.EXTRAP_FIXED, 0.001, 5),
    ("order3_r1", dict(dims=[9, 7, 8], R=1, c=None, eta=1e-3, dtype=np.float64), b.TREE_RESTRUCTURED, b.EXTRAP_NONE, 0.0, 4),
    ("order3_r2_square", dict(dims=[2, 5, 3], R=2, c=0.4, eta=1e-3, dtype=np.float64), b.TREE_STANDARD, b.EXTRAP_FIXED, 0.01, 4),
    ("order6_rest", dict(dims=[5, 6, 4, 5, 4, 5], R=3, c=None, eta=1e-3, dtype=np.float64), b.TREE_RESTRUCTURED, b.EXTRAP_FIXED, 0.01, 6),
    ("order6_std", dict(dims=[6, 5, 5, 4, 6, 4], R=4, c=0.3, eta=1e-3, dtype=np.float32), b.TREE_STANDARD, b.EXTRAP_NONE, 0.0, 4),
]


def _krp_split_count(dims, R, tree, sweeps):
    """Expected split-route Khatri-Rao QRs on the Gram route at order >= 4: every update after the
    first (no update repeats the mode of the one before it, so each has a W formed one update
    ahead)."""
    ops, _ = b.cp_als_qr_schedule(dims, R, tree, sweeps)
    ups = [int(o[1]) for o in ops if int(o[0]) == 1]
    assert all(ups[j] != ups[j - 1] for j in range(1, len(ups)))
    return len(ups) - 1


@pytest.mark.parametrize("route", [b.QR_GRAM, b.QR_HOUSEHOLDER], ids=["gram", "householder"])
@pytest.mark.parametrize("name,cfg,tree,extrap,beta,sweeps", CASES, ids=[c[0] for c in CASES])
def test_fp64_solver_matches_oracle(name, cfg, tree, extrap, beta, sweeps, route):
    """Both QR routes of a sweep against the oracle (Householder QRs throughout); on these
    well-conditioned problems the Gram route's guard never hands a QR to the Householder QR.
    Q_n R_n reproduces A_n to 5e-15 (unit columns): the Gram route's R is the triangle its
    substitution implies, so its backward error is FP64 rounding plus O(E^2), like Householder."""
    cfg = dict(cfg)
    prob = inputs.make_problem(name, cfg.pop("dims"), cfg.pop("R"), seed=3, **cfg)
    fits, A, lam, Q, Rn, st = _run_gpu(prob, tree, extrap, beta, sweeps, route=route)
    ref = _run_oracle(prob, tree, extrap, beta, sweeps)
    assert np.max(np.abs(fits - np.array(ref.fits))) <= 1e-10, (fits, ref.fits)
    for n in range(len(prob.dims)):
        assert o.subspace_sine(A[n], ref.A[n]) <= 1e-10
        assert np.allclose(A[n], ref.A[n], atol=1e-8)
        assert np.abs(Q[n].T @ Q[n] - np.eye(prob.R)).max() < 1e-13
        assert np.abs(Q[n] @ Rn[n] - A[n]).max() < 5e-15
        assert np.all(np.diag(Rn[n]) > 0)
    assert np.allclose(lam, ref.lam, rtol=1e-8)
    assert st.ttm_flops == ref.flops
    assert st.qr_fallbacks == 0
    split = _krp_split_count(prob.dims, prob.R, tree, sweeps)
    assert st.krp_split == (split if route == b.QR_GRAM and len(prob.dims) >= 4 else 0)


@pytest.mark.parametrize("route", [b.QR_GRAM, b.QR_HOUSEHOLDER], ids=["gram", "householder"])
def test_factor_qr_guard_hands_collinear_factor_to_householder(route):
    """Mode 0's true factor has two columns 1e-7 apart (kappa(A_0) ~ 1e7, so the Gram route's
    orthogonality correction would be ~1e-2): its factor QR must go to the Householder QR, while
    the other modes' (well-conditioned) QRs stay on the Gram route.  Both routes track the
    oracle; the least-squares problems themselves stay well-conditioned (the Khatri-Rao Grams
    of the other modes are), so the fit and every normalised factor agree to rounding."""
    dims, R, seed = [30, 28, 26], 5, 11
    B = inputs.gaussian_factors(dims, R, seed)
    g = np.random.default_rng(seed)
    B[0][:, 1] = B[0][:, 0] + 1e-7 * g.standard_normal(dims[0])
    X = inputs.add_noise(inputs.cp_dense(B), 1e-6, seed)
    prob = inputs.Problem("collinear_mode0", dims, R, np.ascontiguousarray(X), inputs.init_factors(dims, R, seed),
                          B, 1e-6, seed)
    sweeps = 4
    fits, A, lam, Q, Rn, st = _run_gpu(prob, b.TREE_RESTRUCTURED, b.EXTRAP_NONE, 0.0, sweeps, route=route)
    ref = _run_oracle(prob, b.TREE_RESTRUCTURED, b.EXTRAP_NONE, 0.0, sweeps)
    assert np.linalg.cond(A[0]) > 1e6
    assert np.max(np.abs(fits - np.array(ref.fits))) <= 1e-10, (fits, ref.fits)
    for n in range(3):
        assert np.allclose(A[n], ref.A[n], atol=1e-8), (n, np.abs(A[n] - ref.A[n]).max())
        assert np.abs(Q[n].T @ Q[n] - np.eye(R)).max() < 1e-13
        assert np.allclose(Q[n] @ Rn[n], A[n], atol=1e-13)
    if route == b.QR_GRAM:
        # mode 0's factor QR every sweep; another factor may come close to kappa ~ 1e4 on the way
        # (the guard's 1e-8 on kappa^2 2^-53) and be handed over too
        assert st.qr_fallbacks >= sweeps
    else:
        assert st.qr_fallbacks == 0


@pytest.mark.parametrize("route", [b.QR_GRAM, b.QR_HOUSEHOLDER], ids=["gram", "householder"])
def test_factor_qr_second_cholesky_pass_on_moderately_collinear_factor(route):
    """Mode 0's true factor has two columns 0.03 apart.  From sweep 2 on, ALS drives the mode-0
    iterate to kappa ~ 1e4 .. 1e5 (measured on the oracle), so the first Cholesky pass of its
    Gram-route QR leaves max |E| ~ kappa^2 2^-48 ~ 1e-6 .. 3e-5: above the first-order correction's
    1e-8, below 1e-3.  A second Cholesky pass (CholeskyQR2) must finish those QRs, without the
    Householder QR, and the result must still be the unique QR: fits and factors as the oracle's,
    Q orthonormal and Q R = A to rounding."""
    dims, R, seed = [30, 28, 26], 5, 11
    B = inputs.gaussian_factors(dims, R, seed)
    g = np.random.default_rng(seed)
    B[0][:, 1] = B[0][:, 0] + 0.03 * g.standard_normal(dims[0])
    X = inputs.add_noise(inputs.cp_dense(B), 1e-6, seed)
    prob = inputs.Problem("moderately_collinear_mode0", dims, R, np.ascontiguousarray(X),
                          inputs.init_factors(dims, R, seed), B, 1e-6, seed)
    sweeps = 5
    fits, A, lam, Q, Rn, st = _run_gpu(prob, b.TREE_RESTRUCTURED, b.EXTRAP_NONE, 0.0, sweeps, route=route)
    ref = _run_oracle(prob, b.TREE_RESTRUCTURED, b.EXTRAP_NONE, 0.0, sweeps)
    assert np.linalg.cond(A[0]) > 3e3
    assert np.max(np.abs(fits - np.array(ref.fits))) <= 1e-10, (fits, ref.fits)
    for n in range(3):
        assert np.allclose(A[n], ref.A[n], atol=1e-8), (n, np.abs(A[n] - ref.A[n]).max())
        assert np.abs(Q[n].T @ Q[n] - np.eye(R)).max() < 1e-13
        assert np.allclose(Q[n] @ Rn[n], A[n], atol=1e-13)
        assert np.all(np.diag(Rn[n]) > 0)
    if route == b.QR_GRAM:
        assert st.qr_second_pass >= 3, (st.qr_second_pass, st.qr_fallbacks)
        assert st.qr_fallbacks == 0, (st.qr_second_pass, st.qr_fallbacks)
    else:
        assert st.qr_second_pass == 0 and st.qr_fallbacks == 0


@pytest.mark.parametrize("order", [4, 5])
def test_split_krp_qr_carries_the_guard_of_its_prefetched_half(order):
    """The starting factors of modes 2 .. N-1 have columns 0 and 1 1e-7 apart, so the Khatri-Rao
    product of their triangles has kappa ~ 1e7 (the other modes keep every product that also
    holds one of them well-conditioned).  In the first sweep the QR for mode 1 takes the split
    route: W, the product of the triangles of modes 2 .. N-1, was formed from those starting
    factors one update ahead; its guard must reach the final level so that the whole QR goes to
    the nested Householder QR, like mode 0's QR on the nested route (its first level is the
    same product).  The factors and fits then track the oracle to rounding."""
    dims = [14, 13, 12, 11] if order == 4 else [9, 8, 7, 6, 7]
    R, seed, sweeps = 4, 5, 4
    B = inputs.gaussian_factors(dims, R, seed)
    X = inputs.add_noise(inputs.cp_dense(B), 1e-4, seed)
    A0 = inputs.init_factors(dims, R, seed)
    g = np.random.default_rng(seed)
    for n in range(2, order):
        A0[n][:, 1] = A0[n][:, 0] + 1e-7 * g.standard_normal(dims[n])
    prob = inputs.Problem(f"collinear_start_order{order}", dims, R, np.ascontiguousarray(X), A0, B, 1e-4, seed)
    fits, A, lam, Q, Rn, st = _run_gpu(prob, b.TREE_RESTRUCTURED, b.EXTRAP_NONE, 0.0, sweeps)
    ref = _run_oracle(prob, b.TREE_RESTRUCTURED, b.EXTRAP_NONE, 0.0, sweeps)
    assert np.max(np.abs(fits - np.array(ref.fits))) <= 1e-10, (fits, ref.fits)
    for n in range(len(dims)):
        assert o.subspace_sine(A[n], ref.A[n]) <= 1e-10
        assert np.allclose(A[n], ref.A[n], atol=1e-8), (n, np.abs(A[n] - ref.A[n]).max())
        assert np.abs(Q[n].T @ Q[n] - np.eye(R)).max() < 1e-13
    assert st.krp_split == _krp_split_count(dims, R, b.TREE_RESTRUCTURED, sweeps)
    # mode 0's nested QR and mode 1's split QR of the first sweep (the starting QRs are Householder)
    assert st.qr_fallbacks >= 2, st.qr_fallbacks


def test_cube60_fifty_sweeps_parity():
    """The 60^3 FP64 rank-5 workload, standard tree, 50 sweeps: fit and factor subspaces <= 1e-10."""
    prob = inputs.workload("cube60_r5_f64", seed=0)
    fits, A, lam, Q, Rn, st = _run_gpu(prob, b.TREE_STANDARD, b.EXTRAP_NONE, 0.0, 50)
    ref = _run_oracle(prob, b.TREE_STANDARD, b.EXTRAP_NONE, 0.0, 50)
    assert np.max(np.abs(fits - np.array(ref.fits))) <= 1e-10
    for n in range(3):
        assert o.subspace_sine(A[n], ref.A[n]) <= 1e-10
        assert np.allclose(Q[n].T @ Q[n], np.eye(5), atol=1e-13)
    assert fits[-1] > 0.9998


MIXED = [
    ("mixed_order3", dict(dims=[40, 36, 33], R=8, c=0.5, eta=1e-2), b.TREE_RESTRUCTURED, b.EXTRAP_FIXED, 0.01, 8),
    ("mixed_order4", dict(dims=[14, 12, 13, 11], R=5, c=0.3, eta=1e-2), b.TREE_RESTRUCTURED, b.EXTRAP_NONE, 0.0, 6),
    ("mixed_order5", dict(dims=[8, 7, 9, 8, 7], R=4, c=None, eta=1e-2), b.TREE_STANDARD, b.EXTRAP_FIXED, 0.01, 5),
    ("mixed_order6", dict(dims=[8, 6, 8, 5, 6, 8], R=4, c=None, eta=1e-2), b.TREE_RESTRUCTURED, b.EXTRAP_NONE, 0.0, 5),
]


@pytest.mark.parametrize("name,cfg,tree,extrap,beta,sweeps", MIXED, ids=[c[0] for c in MIXED])
def test_split_precision_solver_tracks_oracle(name, cfg, tree, extrap, beta, sweeps):
    """Mixed path (split-bf16 TTMs at every tree level, FP64 QRs): per-sweep fit and factor
    subspaces against the FP64 oracle on the same FP32 tensor.  Each split level carries ~2^-17
    relative operand error; two levels times the conditioning of the Hadamard Grams of
    congruence-0.5 rank-8 factors (kappa ~ 9) give ~1.4e-4.  The bound per sweep is 1e-4 for the
    fit and 3e-4 for the subspaces, or 10x the oracle's own change there when X is perturbed by a
    random 2^-16 relative amount (the split operands' error), whichever is larger: sides that are
    not multiples of 8 run every TTM over X on the tensor cores through the padded split copy (one
    more split level), and a sweep on a steep stretch of the fit curve moves by more."""
    cfg = dict(cfg)
    prob = inputs.make_problem(name, cfg.pop("dims"), cfg.pop("R"), seed=4, dtype=np.float32, **cfg)
    fits, A, lam, Q, Rn, st = _run_gpu(prob, tree, extrap, beta, sweeps, prec=b.PREC_SPLIT_BF16)
    ref = _run_oracle(prob, tree, extrap, beta, sweeps)
    g = np.random.default_rng(1)
    pert = inputs.Problem(prob.name, prob.dims, prob.R,
                          prob.X.astype(np.float64) * (1.0 + 2.0 ** -16 * g.standard_normal(prob.X.shape)),
                          prob.A0, prob.true_factors, prob.eta, prob.seed)
    ref_p = _run_oracle(pert, tree, extrap, beta, sweeps)
    fit_tol = np.maximum(1e-4, 10 * np.abs(np.array(ref_p.fits) - np.array(ref.fits)))
    assert np.all(np.abs(fits - np.array(ref.fits)) <= fit_tol), (fits, ref.fits, fit_tol)
    for n in range(len(prob.dims)):
        sub_tol = max(3e-4, 10 * o.subspace_sine(ref_p.A[n], ref.A[n]))
        assert o.subspace_sine(A[n], ref.A[n]) <= sub_tol, (n, sub_tol)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_fit_exact_matches_dense_residual(dtype):
    """cp_als_qr_fit_exact against the oracle's dense ||X - [[lambda; A]]|| with the GPU's own factors."""
    prob = inputs.make_problem("fx", [31, 29, 33], 6, seed=12, c=0.4, eta=3e-3, dtype=dtype)
    X = _dev(prob.X)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_FP64, extrap=b.EXTRAP_NONE)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), dtype == np.float64, prob.A0, opts) as d:
        fits = d.sweep(15)
        A, lam, _, _ = d.factors()
        fx = d.fit_exact()
    ref = o.fit_explicit(prob.X, lam, A)
    assert abs(fx - ref) <= 1e-8
    assert abs(fits[-1] - ref) <= 1e-8


@pytest.mark.parametrize("dims,R", [([37, 29, 36], 6), ([20, 30, 260], 8), ([36, 33, 40, 64], 32),
                                    ([6, 5, 7, 4, 8], 4), ([3, 4, 8], 3), ([150, 130, 128], 16)])
def test_fit_exact_tensor_core_residual(dims, R):
    """FP32 tensors whose last dimension is a multiple of 4 take the tensor-core residual (3xTF32).
    A last side below 128 takes the modes before it into the columns: 29 x 36 = 1044 columns in
    five ragged groups over one ragged row tile, 40 x 64 at order 4 with R = 32, three modes
    folded (7 x 4 x 8) at order 5, every mode but the first folded (4 x 8, three rows); unfolded:
    two column groups (I_last = 260), and 128 columns over 150 x 130 rows.  Fit against the
    oracle's dense residual."""
    prob = inputs.make_problem("fxtc", dims, R, seed=13, c=0.5, eta=2e-3, dtype=np.float32)
    X = _dev(prob.X)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_FP64, extrap=b.EXTRAP_NONE)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
        d.sweep(6)
        A, lam, _, _ = d.factors()
        fx = d.fit_exact()
    ref = o.fit_explicit(prob.X, lam, A)
    assert abs(fx - ref) <= 1e-8


@pytest.mark.parametrize("extrap,beta", [(b.EXTRAP_PAPER, 0.0), (b.EXTRAP_FIXED, 0.01), (b.EXTRAP_NONE, 0.0)])
def test_lagged_fit_equals_sweep_by_sweep_fit(extrap, beta):
    """Split path: cp_als_qr_sweep reads the explicit-residual fit of a sweep one sweep late once
    beta no longer depends on the fit (the residual runs beside the next sweep's first factor
    QR).  Fits, betas and factors equal those of sweep-by-sweep reads (cp_als_qr_sweep(1) per
    sweep), up to the summation order of the residual's CTA partials."""
    prob = inputs.make_problem("lag", [48, 40, 56], 8, seed=9, c=0.6, eta=1e-3, dtype=np.float32)
    X = _dev(prob.X)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_SPLIT_BF16, extrap=extrap, beta_fixed=beta)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
        f_many = d.sweep(12)
        A1, lam1, _, _ = d.factors()
        h1 = d.history()
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
        f_one = np.array([d.sweep(1)[0] for _ in range(12)])
        A2, lam2, _, _ = d.factors()
        h2 = d.history()
    assert np.all(np.isfinite(f_many))
    assert np.allclose(f_many, f_one, rtol=0, atol=1e-12), (f_many, f_one)
    assert np.array_equal(h1[1], h2[1])  # betas
    for a1, a2 in zip(A1, A2):
        assert np.array_equal(a1, a2)
    assert np.array_equal(lam1, lam2)


def test_lagged_fit_of_a_small_tensor_after_a_large_one():
    """The lagged residual runs as clusters over all but one GPC; a tensor with fewer row tiles than
    those CTAs leaves most of them without work.  Their partial-sum slots must not enter the fit:
    a large tensor's lagged sweeps first fill every slot of a workspace that the small tensor's
    context may then reuse, and the small tensor's lagged fits must still equal its
    sweep-by-sweep fits."""
    big = inputs.make_problem("lag_big", [160, 150, 144], 8, seed=3, c=0.5, eta=1e-3, dtype=np.float32)
    small = inputs.make_problem("lag_small", [30, 28, 24], 6, seed=9, c=0.6, eta=1e-2, dtype=np.float32)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_SPLIT_BF16, extrap=b.EXTRAP_FIXED, beta_fixed=0.01)
    Xb = _dev(big.X)
    with b.Decomposition(big.dims, big.R, Xb.data_ptr(), False, big.A0, opts) as d:
        d.sweep(6)
    del Xb
    Xs = _dev(small.X)
    with b.Decomposition(small.dims, small.R, Xs.data_ptr(), False, small.A0, opts) as d:
        f_many = d.sweep(12)
        lagged = d.stats().lagged_fits
    with b.Decomposition(small.dims, small.R, Xs.data_ptr(), False, small.A0, opts) as d:
        f_one = np.array([d.sweep(1)[0] for _ in range(12)])
    assert lagged >= 1
    assert np.allclose(f_many, f_one, rtol=0, atol=1e-12), (f_many - f_one)


@pytest.mark.parametrize("delta", [1e-2, 1e-4, 1e-10, 0.0])
def test_krp_qr_gram_route_falls_back_on_ill_conditioned_products(delta):
    """The Khatri-Rao QR of two triangles goes through the Gram matrix (Cholesky of the Hadamard
    product of the triangles' Grams, one orthogonality correction); when the correction is not
    small it is finished by a second Cholesky pass or, for a failed pivot or a larger E, by the
    Householder QR.  Columns 0 and 1 of both source matrices are delta apart (a singular Gram at
    delta = 0): whichever finishes it, the result must be the unique QR, orthonormal and
    reproducing Z to rounding, with R as the oracle's up to the QR's perturbation bound
    (kappa(Z) times the rounding unit)."""
    R = 12
    g = np.random.default_rng(77)
    tri = []
    for _ in range(2):
        B = g.standard_normal((R + 6, R))
        B[:, 1] = B[:, 0] + delta * g.standard_normal(R + 6)
        Rk = o.householder_qr(B)[1]
        tri.append(Rk)
    Z = o.khatri_rao(tri)
    Q0 = torch.empty(Z.shape, dtype=torch.float64, device=DEV)
    R0 = torch.empty((R, R), dtype=torch.float64, device=DEV)
    Rd = _dev(np.stack(tri))
    b.cpqr_krp_qr(Rd.data_ptr(), 2, R, Q0.data_ptr(), R0.data_ptr())
    torch.cuda.synchronize()
    Qg, Rg = Q0.cpu().numpy(), R0.cpu().numpy()
    assert np.abs(Qg.T @ Qg - np.eye(R)).max() < 1e-13
    assert np.abs(Qg @ Rg - Z).max() < 1e-13 * np.abs(Z).max()
    assert np.all(np.diag(Rg)[np.abs(np.diag(Rg)) > 1e-12] > 0)
    if delta > 0:
        Q0r, R0r = o.householder_qr(Z)
        tol = max(1e-12, 1e-15 * np.linalg.cond(Z))
        assert np.allclose(Rg, R0r, atol=tol * np.abs(R0r).max()), (np.abs(Rg - R0r).max(), np.linalg.cond(Z))


CONVERGED_MIXED = [
    ("br_c03", dict(c=0.3), b.EXTRAP_NONE, 0.0, 60),
    ("bre_fixed_c05", dict(c=0.5), b.EXTRAP_FIXED, 0.01, 90),
]


@pytest.mark.parametrize("name,cfg,extrap,beta,sweeps", CONVERGED_MIXED, ids=[c[0] for c in CONVERGED_MIXED])
def test_split_precision_final_fit_within_1e6_of_oracle(name, cfg, extrap, beta, sweeps):
    """Mixed precision at its stated tolerance: on 96^3, R = 16 (FP32 tensor, noise 1e-3) both the
    split path and the FP64 oracle run the restructured tree from the same start for enough
    sweeps to converge (the oracle's last fit change is checked below 1e-10); the final fits,
    each from an explicit residual of its own factors, agree to 1e-6 relative.  At a least-squares
    optimum (beta = 0) the fit is stationary in the factors, so the split operands' ~2^-17 random
    error enters it only to second order.  At eq. 19's scaled fixed point (beta > 0) a relative
    scale error of the model moves the fit to first order: this case holds only because neither
    the split TTMs nor the residual pass are biased (see the bias tests)."""
    prob = inputs.make_problem(name, [96, 96, 96], 16, seed=7, eta=1e-3, dtype=np.float32, **cfg)
    X = _dev(prob.X)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_SPLIT_BF16, extrap=extrap, beta_fixed=beta)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
        fits = d.sweep(sweeps)
        fx = d.fit_exact()
    kw = dict(extrapolate=False) if extrap == b.EXTRAP_NONE else dict(extrapolate=True, beta_fixed=beta)
    ref = o.cp_als_qr(prob.X, prob.R, prob.A0, tree=o.TREE_RESTRUCTURED, max_sweeps=sweeps, **kw)
    assert abs(ref.fits[-1] - ref.fits[-2]) < 1e-10
    f_ref = o.fit_explicit(prob.X, ref.lam, ref.A)
    assert abs(fx - f_ref) / f_ref <= 1e-6, (fx, f_ref)
    assert abs(fits[-1] - f_ref) / f_ref <= 1e-6, (fits[-1], f_ref)
    assert np.max(np.abs(fits - np.array(ref.fits))) <= 1e-4


def test_eq18_plain_extrapolation_alpha_one_matches_oracle():
    """alpha = 1 turns eq. 19 into eq. 18 (Q0^ = Q0 + beta (Q0 - Q0^{k-1})): FP64 path against the
    oracle with the same alpha, fits and factor subspaces within 1e-10."""
    prob = inputs.make_problem("eq18", [21, 19, 23], 5, seed=8, c=0.6, eta=1e-3, dtype=np.float64)
    X = _dev(prob.X)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_FP64, extrap=b.EXTRAP_FIXED, beta_fixed=0.05,
                          alpha=1.0)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), True, prob.A0, opts) as d:
        fits = d.sweep(8)
        A, lam, _, _ = d.factors()
    ref = o.cp_als_qr(prob.X, prob.R, prob.A0, tree=o.TREE_RESTRUCTURED, extrapolate=True, beta_fixed=0.05,
                      alpha=1.0, max_sweeps=8)
    other = o.cp_als_qr(prob.X, prob.R, prob.A0, tree=o.TREE_RESTRUCTURED, extrapolate=True, beta_fixed=0.05,
                        max_sweeps=8)
    assert np.max(np.abs(fits - np.array(ref.fits))) <= 1e-10
    assert np.max(np.abs(np.array(other.fits) - np.array(ref.fits))) > 1e-6  # alpha matters here
    for n in range(3):
        assert o.subspace_sine(A[n], ref.A[n]) <= 1e-10


@pytest.mark.parametrize("prec", [b.PREC_FP64, b.PREC_SPLIT_BF16], ids=["fp64", "split"])
def test_bre_with_beta_zero_is_br_bit_for_bit(prec):
    """beta = 0 in eq. 19 leaves Q0 as it is: ALS-QR-BRE with a fixed beta of 0 runs the same
    kernels on the same data as ALS-QR-BR, so fits and factors agree bit for bit."""
    prob = inputs.make_problem("br0", [32, 24, 40], 6, seed=9, c=0.4, eta=1e-3, dtype=np.float32)
    X = _dev(prob.X)
    out = []
    for ex in (b.EXTRAP_NONE, b.EXTRAP_FIXED):
        opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=prec, extrap=ex, beta_fixed=0.0)
        with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
            fits = np.array([d.sweep(1)[0] for _ in range(6)])
            A, lam, _, _ = d.factors()
        out.append((fits, A, lam))
    assert np.array_equal(out[0][0], out[1][0])
    for a0, a1 in zip(out[0][1], out[1][1]):
        assert np.array_equal(a0, a1)


def test_paper_rule_and_fixed_beta_follow_the_oracle():
    """The Section 4.2 rule (beta switched on by the fit change, banded by the fit) against a
    fixed beta from the second sweep, FP64 path, both against the oracle to 1e-10: the rule's
    activation sweep and band match the oracle's, and the two controllers give different runs."""
    prob = inputs.make_problem("rule", [26, 22, 24], 6, seed=10, c=0.7, eta=1e-3, dtype=np.float64)
    X = _dev(prob.X)
    res = {}
    for name, ex, beta in (("rule", b.EXTRAP_PAPER, 0.0), ("fixed", b.EXTRAP_FIXED, 0.002)):
        opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_FP64, extrap=ex, beta_fixed=beta)
        with b.Decomposition(prob.dims, prob.R, X.data_ptr(), True, prob.A0, opts) as d:
            fits = d.sweep(12)
            hist = d.history()
        kw = dict(extrapolate=True) if ex == b.EXTRAP_PAPER else dict(extrapolate=True, beta_fixed=beta)
        ref = o.cp_als_qr(prob.X, prob.R, prob.A0, tree=o.TREE_RESTRUCTURED, max_sweeps=12, **kw)
        assert np.max(np.abs(fits - np.array(ref.fits))) <= 1e-10, name
        assert np.array_equal(hist[1], np.array(ref.betas)), name
        res[name] = ref
    assert any(bb > 0 for bb in res["rule"].betas)  # the rule activates within these sweeps
    assert res["rule"].betas != res["fixed"].betas


def test_fit_exact_at_an_extrapolated_fixed_point():
    """At eq. 19's fixed point the model is the least-squares model scaled by 1 + beta (1 - alpha),
    so the residual is no longer orthogonal to it and a relative scale error e of the residual
    pass's model entries moves the fit by about e (at a least-squares optimum it would not move it
    at all).  The FP64 path (factors equal to the oracle's to 1e-15) after 90 sweeps with a fixed
    beta of 0.01: cp_als_qr_fit_exact against the oracle's dense residual of the same factors to
    1.5e-7 (truncating TF32 splits gave 5.6e-7)."""
    prob = inputs.make_problem("fx_bre", [96, 96, 96], 16, seed=7, c=0.5, eta=1e-3, dtype=np.float32)
    X = _dev(prob.X)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_FP64, extrap=b.EXTRAP_FIXED, beta_fixed=0.01)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
        fits = d.sweep(90)
        A, lam, _, _ = d.factors()
        fx = d.fit_exact()
    ref = o.fit_explicit(prob.X, lam, A)
    assert abs(fx - ref) <= 1.5e-7, (fx, ref)
    assert abs(fits[-1] - ref) <= 1e-9  # the reduced form is exact here
