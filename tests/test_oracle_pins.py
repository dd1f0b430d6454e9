"""Pins of the oracle's checking helpers and of the learned proposer's oracle network against
values worked out by hand (not against the oracle itself).

* mlp_oracle.forward / loss_and_grad: a network with a handful of non-zero weights whose
  logits follow from the layer equations by hand (a dropped bias, a transposed weight matrix or
  a missing ReLU changes them);
* mlp_oracle.adam_step: two steps of Adam (Kingma & Ba, 2015, Algorithm 1) on one scalar, every
  intermediate written out;
* cpqr_oracle.subspace_sine: two planes at a constructed principal angle theta;
* cpqr_oracle.factor_match_score: permuted and scaled copies of the factors score 1, factors
  orthogonal to the truth score 0, and known cosines give their product.
"""
import math

import numpy as np
import pytest

from oracle import cpqr_oracle as o
from oracle import mlp_oracle as m


def _sparse_network():
    """Layer l: z = W_l h + b_l, ReLU on the hidden layers.  Non-zero parameters:
    W0[2, 5] = 2, b0[2] = -1;  W1[7, 2] = 3, b1[7] = 0.5;  W2[1, 7] = 0.5, b2[1] = 1, b2[4] = 2;
    W3[c, 1] = c, W3[c, 4] = -1, b3[c] = c / 4."""
    layers = [(np.zeros((o_, i_)), np.zeros(o_)) for o_, i_ in m.SHAPES]
    layers[0][0][2, 5], layers[0][1][2] = 2.0, -1.0
    layers[1][0][7, 2], layers[1][1][7] = 3.0, 0.5
    layers[2][0][1, 7], layers[2][1][1], layers[2][1][4] = 0.5, 1.0, 2.0
    for c in range(m.C):
        layers[3][0][c, 1], layers[3][0][c, 4], layers[3][1][c] = float(c), -1.0, c / 4.0
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def test_forward_of_a_network_evaluated_by_hand():
    p = _sparse_network()
    g = np.random.default_rng(0)
    X = g.standard_normal((2, m.F))  # every feature but 5 is ignored by the network
    X[0, 5], X[1, 5] = 3.0, -3.0
    logits, _ = m.forward(p, X)
    # x5 = 3:  h0[2] = relu(2*3 - 1) = 5;  h1[7] = relu(3*5 + 0.5) = 15.5;
    #          h2[1] = relu(0.5*15.5 + 1) = 8.75, h2[4] = relu(2) = 2;  z_c = 8.75 c - 2 + c/4 = 9 c - 2
    # x5 = -3: h0[2] = relu(-7) = 0;  h1[7] = relu(0.5) = 0.5;
    #          h2[1] = relu(0.25 + 1) = 1.25, h2[4] = 2;  z_c = 1.25 c - 2 + c/4 = 1.5 c - 2
    c = np.arange(m.C)
    assert np.array_equal(logits[0], 9.0 * c - 2.0)
    assert np.array_equal(logits[1], 1.5 * c - 2.0)


def test_loss_of_a_network_evaluated_by_hand():
    p = _sparse_network()
    X = np.zeros((1, m.F))
    X[0, 5] = -3.0
    # z_c = 1.5 c - 2 (above); label 3: loss = log sum_c exp(1.5 c - 2) - (1.5 * 3 - 2)
    want = math.log(sum(math.exp(1.5 * c - 2.0) for c in range(m.C))) - 2.5
    loss, _ = m.loss_and_grad(p, X, [3])
    assert abs(loss - want) < 1e-14


def test_adam_two_steps_by_hand():
    """w0 = 1, m0 = v0 = 0, lr = 0.1, beta1 = 0.9, beta2 = 0.999, eps = 1e-8; g1 = 0.5, g2 = -1.
    Step 1: m1 = 0.05, v1 = 0.00025, m^ = 0.05 / 0.1 = 0.5, v^ = 0.00025 / 0.001 = 0.25,
            w1 = 1 - 0.1 * 0.5 / (0.5 + 1e-8) = 0.900000002 (to 1e-16).
    Step 2: m2 = 0.9 * 0.05 - 0.1 = -0.055, v2 = 0.999 * 0.00025 + 0.001 = 0.00124975,
            m^ = -0.055 / 0.19 = -11/38, v^ = 0.00124975 / 0.001999 = 4999/7996,
            w2 = w1 + 0.1 * (11/38) / (sqrt(4999/7996) + 1e-8)."""
    w, mm, v = np.array([1.0]), np.zeros(1), np.zeros(1)
    w, mm, v = m.adam_step(w, mm, v, np.array([0.5]), 0.1, 1)
    assert abs(mm[0] - 0.05) < 1e-16 and abs(v[0] - 0.00025) < 1e-18  # 1 - 0.9 rounds in FP64
    assert abs(w[0] - 0.900000002) < 1e-15
    w, mm, v = m.adam_step(w, mm, v, np.array([-1.0]), 0.1, 2)
    assert abs(mm[0] + 0.055) < 1e-16 and abs(v[0] - 0.00124975) < 1e-17
    w2 = 0.900000002 + 0.1 * (11 / 38) / (math.sqrt(4999 / 7996) + 1e-8)
    assert abs(w[0] - w2) < 1e-15
    assert abs(w[0] - 0.93661035424) < 1e-11


@pytest.mark.parametrize("theta", [1e-12, 1e-9, 1e-6, 1e-3, 0.1, 0.5])
def test_subspace_sine_of_planes_at_a_constructed_angle(theta):
    """span{e1, e2} against span{cos(theta) e1 + sin(theta) e3, e2}, both rotated by the same random
    orthogonal matrix and given in non-orthogonal bases: the largest principal angle is theta."""
    g = np.random.default_rng(int(theta * 1e12) % 1000)
    n = 9
    U = np.linalg.qr(g.standard_normal((n, n)))[0]
    E = np.eye(n)
    A = U @ np.stack([E[0], E[1]], axis=1)
    B = U @ np.stack([math.cos(theta) * E[0] + math.sin(theta) * E[2], E[1]], axis=1)
    Ma = np.array([[2.0, 1.0], [0.5, 1.5]])
    Mb = np.array([[1.0, -0.7], [0.3, 2.0]])
    s = o.subspace_sine(A @ Ma, B @ Mb)
    assert abs(s - math.sin(theta)) <= 1e-15 + 1e-3 * math.sin(theta), (s, math.sin(theta))
    assert o.subspace_sine(A @ Ma, A @ Mb) < 1e-15


def test_factor_match_score_known_cases():
    g = np.random.default_rng(4)
    dims, R = [7, 6, 5], 3
    A = [g.standard_normal((d, R)) for d in dims]
    perm = [2, 0, 1]
    scaled = [a[:, perm] * np.array([-2.0, 0.5, 3.0])[None, :] for a in A]
    assert abs(o.factor_match_score(A, scaled) - 1.0) < 1e-14
    # orthogonal in one mode: every product of cosines holds a zero factor
    Q = np.linalg.qr(g.standard_normal((dims[0], 2 * R)))[0]
    A_true = [Q[:, :R]] + A[1:]
    A_orth = [Q[:, R:]] + A[1:]
    assert o.factor_match_score(A_true, A_orth) < 1e-14
    # one component rotated by a known angle in one mode: its term is cos(phi), the others 1
    phi = 0.3
    Q3 = np.linalg.qr(g.standard_normal((dims[0], R + 1)))[0]
    A_t = [Q3[:, :R]] + [np.eye(d)[:, :R] for d in dims[1:]]
    rot = Q3[:, :R].copy()
    rot[:, 1] = math.cos(phi) * Q3[:, 1] + math.sin(phi) * Q3[:, R]
    A_e = [rot] + [np.eye(d)[:, :R] for d in dims[1:]]
    assert abs(o.factor_match_score(A_t, A_e) - (2 + math.cos(phi)) / 3) < 1e-14
