"""Pins of the oracle MLP: analytic gradient against central finite differences and the
loss of a zero network (uniform softmax = log C)."""
import numpy as np

from oracle import mlp_oracle as m


def test_zero_network_loss_is_log_c():
    X = np.random.default_rng(0).standard_normal((5, m.F))
    loss, _ = m.loss_and_grad(np.zeros(m.NPARAMS), X, [0, 1, 2, 3, 4])
    assert abs(loss - np.log(m.C)) < 1e-15


def test_gradient_matches_finite_differences():
    g = np.random.default_rng(1)
    p = m.init_params(3) * 0.5 + 0.01 * g.standard_normal(m.NPARAMS)
    X = g.standard_normal((6, m.F))
    y = g.integers(0, m.C, 6)
    _, grad = m.loss_and_grad(p, X, y)
    idx = np.concatenate([g.choice(m.NPARAMS, 60, replace=False), [0, m.NPARAMS - 1, m.NPARAMS - 9]])
    h = 1e-6
    for i in idx:
        e = np.zeros(m.NPARAMS)
        e[i] = h
        fd = (m.loss_and_grad(p + e, X, y)[0] - m.loss_and_grad(p - e, X, y)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, grad[i])


def test_parameter_count_and_layout():
    assert m.NPARAMS == 32 * 128 + 128 + 2 * (128 * 128 + 128) + 128 * 8 + 8
    layers = m.unpack(np.arange(m.NPARAMS, dtype=float))
    assert layers[0][0][0, 1] == 1.0 and layers[0][1][0] == 128 * 32


def test_bf16_rounding_definition():
    vals = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 65504.0, 1e-30], dtype=np.float32)
    r = m.bf16(vals)
    # bf16 keeps 8 significand bits: spacing 2^-7 in [1, 2)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125
    assert abs(r[3] + 3.140625) < 1e-12
    assert np.all(np.abs(r - vals) <= np.abs(vals) * 2 ** -8)
