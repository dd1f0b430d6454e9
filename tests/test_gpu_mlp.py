"""GPU kernels of the learned proposer against the FP64 oracle network, the feature
definition, checkpoint / rollback of the solver and the learned-extrapolation sweep."""
import math

import numpy as np
import pytest

from oracle import cpqr_oracle as o
from oracle import mlp_oracle as mo
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


bf16_round = mo.bf16


def _t(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dt)


@pytest.mark.parametrize("B", [1, 7, 256])
def test_forward_and_gradient_match_oracle(B):
    g = np.random.default_rng(B)
    params = (mo.init_params(1) + 0.01 * g.standard_normal(mo.NPARAMS)).astype(np.float32)
    X = g.standard_normal((B, mo.F)).astype(np.float32)
    y = g.integers(0, mo.C, B).astype(np.int32)
    pd, Xd, yd = _t(params), _t(X), _t(y, torch.int32)
    work = torch.empty(b.cpqr_mlp_work_bytes(B), dtype=torch.uint8, device=DEV)
    logits = torch.empty((B, mo.C), dtype=torch.float32, device=DEV)
    grad = torch.empty(mo.NPARAMS, dtype=torch.float32, device=DEV)
    loss = torch.empty(1, dtype=torch.float32, device=DEV)
    b.cpqr_mlp_forward(pd.data_ptr(), Xd.data_ptr(), B, logits.data_ptr(), work.data_ptr())
    b.cpqr_mlp_grad(pd.data_ptr(), Xd.data_ptr(), yd.data_ptr(), B, grad.data_ptr(), loss.data_ptr(),
                    work.data_ptr())
    torch.cuda.synchronize()
    # The network's weights, inputs and stored hidden activations are bf16 and its products
    # accumulate in FP32; the oracle takes the same bf16 weights and inputs, rounds its stored
    # activations to bf16 at the same points and computes everything else in FP64 (biases are
    # kept in FP32 by the kernels: give the oracle those, not bf16 ones).
    p64 = bf16_round(params)
    for l, (o_, i_) in enumerate(mo.SHAPES):
        off = sum(o * i + o for o, i in mo.SHAPES[:l]) + o_ * i_
        p64[off:off + o_] = params[off:off + o_]
    ref_logits, _ = mo.forward(p64, bf16_round(X), store=mo.bf16)
    ref_loss, ref_grad = mo.loss_and_grad(p64, bf16_round(X), y, store=mo.bf16)
    got = logits.cpu().numpy()
    assert np.max(np.abs(got - ref_logits)) <= 1e-2 * max(1.0, np.max(np.abs(ref_logits)))
    assert abs(loss.item() - ref_loss) <= 1e-3 * max(1.0, ref_loss)
    gg = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - ref_grad) <= 1e-2 * np.linalg.norm(ref_grad)
    # against unrounded FP64 activations the bf16 storage costs a few percent at batch >= 7
    if B >= 7:
        _, g64 = mo.loss_and_grad(p64, bf16_round(X), y)
        assert np.linalg.norm(gg - g64) <= 6e-2 * np.linalg.norm(g64)


def test_adam_matches_oracle():
    g = np.random.default_rng(5)
    w = g.standard_normal(mo.NPARAMS).astype(np.float32)
    gr = g.standard_normal(mo.NPARAMS).astype(np.float32)
    m0 = np.zeros(mo.NPARAMS, np.float32)
    v0 = np.zeros(mo.NPARAMS, np.float32)
    wd, md, vd, gd = _t(w), _t(m0), _t(v0), _t(gr)
    ref = (w.astype(np.float64), m0.astype(np.float64), v0.astype(np.float64))
    for step in (1, 2, 3):
        b.cpqr_mlp_adam(wd.data_ptr(), md.data_ptr(), vd.data_ptr(), gd.data_ptr(), 1e-3, step)
        ref = mo.adam_step(*ref, gr.astype(np.float64), 1e-3, step)
    torch.cuda.synchronize()
    assert np.max(np.abs(wd.cpu().numpy() - ref[0])) < 1e-5


def test_features_follow_their_definition():
    fits = np.array([0.5, 0.7, 0.8, 0.85, 0.86, 0.861, 0.8611, 0.86111, 0.861111, 0.8611111])
    betas = np.array([0, 0, 0, 2e-3, 2e-3, 2e-3, 2e-3, 2e-3, 2e-3, 2e-3])
    f = b.cpqr_mlp_features(fits, betas, 2e-3, True)
    n = len(fits)
    for j in range(8):
        k = n - 1 - j
        assert f[3 * j] == pytest.approx(math.log10(1 - fits[k]) / 12, abs=1e-6)
        d = fits[k] - fits[k - 1]
        assert f[3 * j + 1] == pytest.approx(math.copysign((math.log10(abs(d)) + 14) / 14, d), abs=1e-6)
        assert f[3 * j + 2] == pytest.approx(math.log10(betas[k] + 1e-8) / 8, abs=1e-6)
    assert f[24] == pytest.approx(math.log10(n + 1) / 3, abs=1e-6)
    assert f[25] == pytest.approx(math.log10(2e-3 + 1e-8) / 8, abs=1e-6)
    assert f[26] == 1.0 and np.all(f[27:] == 0)
    short = b.cpqr_mlp_features(fits[:1], betas[:1], 0.0, False)
    assert short[1] == 0 and np.all(short[3:24] == 0)


def _problem(N=3):
    dims = [30, 28, 26] if N == 3 else [14, 12, 13, 11]
    return inputs.make_problem("ck", dims, 6, seed=9, c=0.6, eta=1e-2, dtype=np.float32)


@pytest.mark.parametrize("prec", [b.PREC_FP64, b.PREC_SPLIT_BF16])
@pytest.mark.parametrize("N", [3, 4])
def test_checkpoint_rollback_reproduces_branches(prec, N):
    prob = _problem(N)
    X = _t(prob.X)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=prec, extrap=b.EXTRAP_PAPER)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
        d.sweep(3)
        d.checkpoint()
        a = [d.sweep_beta(0.02) for _ in range(3)]
        A1 = d.factors()[0]
        d.rollback()
        c = [d.sweep_beta(0.0) for _ in range(2)]
        d.rollback()
        a2 = [d.sweep_beta(0.02) for _ in range(3)]
        A2 = d.factors()[0]
        d.commit()
        fits, betas, _, _ = d.history()
    assert np.allclose(a, a2, rtol=0, atol=1e-12)
    for x, y in zip(A1, A2):
        assert np.allclose(x, y, atol=1e-10)
    assert len(fits) == 6 and np.allclose(betas[3:], 0.02)
    assert not np.allclose(a[:2], c)


def test_device_proposer_features_and_logits_follow_their_definitions():
    """The features the device computes after each sweep equal cpqr_mlp_features of the fit / beta
    history, and its logits equal cpqr_mlp_forward on those features (same bf16 rounding, same
    accumulation order); the proposal is their first arg max."""
    prob = _problem(3)
    X = _t(prob.X)
    w = mo.init_params(7).astype(np.float32)
    for prec in (b.PREC_FP64, b.PREC_SPLIT_BF16):
        opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=prec, extrap=b.EXTRAP_LEARNED, mlp_weights=w)
        with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
            for k in range(11):
                d.sweep(1)
                fits, betas, rule, act = d.history()
                f_dev, lg_dev, cls = b.cp_als_qr_mlp_state(d.ctx)
                f_host = b.cpqr_mlp_features(fits, betas, rule, act)
                assert np.allclose(f_dev, f_host, rtol=1e-6, atol=1e-7), (k, f_dev, f_host)
                pd, xd = _t(w), _t(f_dev[None, :].copy())
                lg = torch.empty((1, b.MLP_CLASSES), dtype=torch.float32, device=DEV)
                work = torch.empty(b.cpqr_mlp_work_bytes(1), dtype=torch.uint8, device=DEV)
                b.cpqr_mlp_forward(pd.data_ptr(), xd.data_ptr(), 1, lg.data_ptr(), work.data_ptr())
                torch.cuda.synchronize()
                assert np.allclose(lg_dev, lg.cpu().numpy()[0], rtol=1e-5, atol=1e-5)
                assert cls == int(np.argmax(lg_dev))


def _constant_network(c):
    """A network whose logits are its last-layer biases: it always proposes class c."""
    p = np.zeros(mo.NPARAMS, dtype=np.float32)
    p[-mo.C:] = -1.0
    p[-mo.C + c] = 1.0
    return p


@pytest.mark.parametrize("c", [0, 6])
def test_judge_protocol_replayed_through_the_public_api(c):
    """A network that always proposes class c (beta = 0, or beta = 1e-2) on the split path.  The
    same run replayed by hand through checkpoint / sweep_beta / rollback: a proposal equal to the
    rule's beta runs as is; within a hold after a loss the rule runs; inside an approval window the
    proposal runs as is; else both branches run from one checkpoint and the proposal is kept only
    if its fit is higher.  Wins double the approval window (<= 128) and reset the hold; losses
    reset the approval and start a hold that doubles on consecutive losses (<= 128); a fit drop of
    more than 1e-7 ends an approval.  Fits and betas agree bit for bit."""
    prob = _problem(3)
    X = _t(prob.X)
    w = _constant_network(c)
    beta_c = b.cp_als_qr_mlp_beta(c)
    sweeps = 24
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_SPLIT_BF16, extrap=b.EXTRAP_LEARNED, mlp_weights=w)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
        for _ in range(sweeps):
            d.sweep(1)
        fits_l, betas_l, _, _ = d.history()
        st = d.stats()
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_SPLIT_BF16, extrap=b.EXTRAP_PAPER)
    judged = wins = 0
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
        approved, window, left = -1, 1, 0
        hold_window, hold_left = 1, 0
        for k in range(sweeps):
            fits, betas, rule, act = d.history()
            if len(fits) < 2 or beta_c == rule:
                d.sweep_beta(rule)
                continue
            if hold_left > 0:
                hold_left -= 1
                d.sweep_beta(rule)
                continue
            if approved == c and left > 0:
                left -= 1
                f = d.sweep_beta(beta_c)
                if not f >= fits[-1] - 1e-7:
                    approved, window, left = -1, 1, 0
                continue
            judged += 1
            d.checkpoint()
            fp = d.sweep_beta(beta_c)
            d.rollback()
            fr = d.sweep_beta(rule)
            if fp > fr:
                d.rollback()
                d.sweep_beta(beta_c)
                wins += 1
                approved, window = c, min(2 * window, 128)
                left = window
                hold_window = 1
            else:
                approved, window, left = -1, 1, 0
                hold_left = hold_window
                hold_window = min(2 * hold_window, 128)
            d.commit()
        fits_m, betas_m, _, _ = d.history()
    assert np.array_equal(betas_l, betas_m), (betas_l, betas_m)
    assert np.array_equal(fits_l, fits_m)
    assert st.judged == judged and judged >= 1
    assert st.accepted == wins + st.preapproved


@pytest.mark.parametrize("c", [0, 6])
def test_lagged_learned_sweeps_replay_through_the_public_api(c):
    """Inside one multi-sweep call on the split path the learned proposer's unjudged sweeps read
    their fit one sweep late (once the rule has activated), with the proposal computed on the
    device beside the next sweep, while judged sweeps first complete every pending fit and run both
    branches from one checkpoint.  Whatever was decided, the kept history must be the trajectory of
    its own betas: replaying them one sweep at a time from the same start reproduces every fit bit
    for bit, and the run judged at least once."""
    # last side a multiple of 4: the tensor-core residual (and so the lag) serves this tensor
    prob = inputs.make_problem("lagged", [30, 28, 24], 6, seed=9, c=0.6, eta=1e-2, dtype=np.float32)
    X = _t(prob.X)
    w = _constant_network(c)
    sweeps = 30
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_SPLIT_BF16, extrap=b.EXTRAP_LEARNED, mlp_weights=w)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
        fits_call = d.sweep(sweeps)
        fits_l, betas_l, _, act = d.history()
        st = d.stats()
    assert act, "the rule never activated: no sweep could lag"
    assert np.array_equal(fits_call, fits_l)
    assert st.judged >= 1 and st.proposals >= st.judged
    assert st.lagged_fits >= 1, (st.lagged_fits, st.judged)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_SPLIT_BF16, extrap=b.EXTRAP_PAPER)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
        fits_r = [d.sweep_beta(float(beta)) for beta in betas_l]
    assert np.array_equal(np.array(fits_r), fits_l), (np.array(fits_r) - fits_l, betas_l, st.judged, st.preapproved,
                                                      st.lagged_fits)


def test_learned_sweep_with_a_random_network_is_judged():
    """An untrained network still runs: every accepted proposal keeps the fit from dropping, a
    rejected one is replaced by the Section 4.2 rule's sweep."""
    prob = _problem(3)
    X = _t(prob.X)
    w = mo.init_params(7).astype(np.float32)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_FP64, extrap=b.EXTRAP_LEARNED, mlp_weights=w)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
        fits = d.sweep(12)
        st = d.stats()
        hist, betas, _, _ = d.history()
    # once the rule has activated, any class other than the rule's beta is a proposal
    assert st.proposals >= 1 and st.accepted <= st.proposals
    assert np.allclose(hist, fits)
    assert np.all(np.isfinite(fits))
