"""Pins of the learned-sketch oracle (CPU): central differences, closed forms, invariances.

The network and loss are not in the paper (the paper draws G at random); what fixes them is
their definition in oracle/sketch_net.py. The pins below check that definition against
things other than itself: finite differences for every gradient, a library QR for the
projector loss, closed forms at special points, and the textbook Adam update.
"""

import numpy as np
import pytest

from oracle import sketch_net as SN

SHAPE = (9, 2, 3, 8, 5)   # d_raw, n_coord, n_freq, hidden, s_out


def _case(seed=0, n=30, k=3):
    rng = np.random.default_rng(seed)
    d0 = SN.dims(*SHAPE)[0]
    npar = d0 * 8 + 8 + 8 * 8 + 8 + 8 * 5 + 5
    theta = rng.standard_normal(npar) * 0.5
    attrs = rng.uniform(0.0, 1.0, (n, SHAPE[0]))
    U, _ = np.linalg.qr(rng.standard_normal((n, k)))
    return theta, attrs, U


def test_unpack_covers_every_parameter_once():
    theta, _, _ = _case()
    parts = SN.unpack(theta, SHAPE)
    assert sum(p.size for p in parts) == theta.size
    assert [p.shape for p in parts] == [(19, 8), (8,), (8, 8), (8,), (8, 5), (5,)]


def test_embedding_closed_form_at_half():
    a = np.full((1, 9), 0.5)
    a[0, 2:] = np.arange(7)
    e = SN.embed(a, 2, 4)
    # sin(pi j / 2), cos(pi j / 2) for j = 1..4, for each of the two coordinates
    one = [1, 0, 0, -1, -1, 0, 0, 1]
    assert np.allclose(e[0, :16], one + one, atol=1e-15)
    assert np.array_equal(e[0, 16:], np.arange(7))


def test_projector_loss_matches_library_qr():
    rng = np.random.default_rng(1)
    G = rng.standard_normal((40, 6))
    U, _ = np.linalg.qr(rng.standard_normal((40, 4)))
    L, _ = SN.projector_loss(G, U, 0.0)
    Q, _ = np.linalg.qr(G)
    assert np.isclose(L, 4.0 - np.linalg.norm(Q.T @ U) ** 2, rtol=1e-12)


def test_projector_loss_special_points():
    rng = np.random.default_rng(2)
    U, _ = np.linalg.qr(rng.standard_normal((25, 3)))
    # U inside range(G): zero loss, zero gradient
    G = np.concatenate([U @ rng.standard_normal((3, 3)), rng.standard_normal((25, 2))], axis=1)
    L, dG = SN.projector_loss(G, U, 0.0)
    assert abs(L) < 1e-20 + 1e-12 and np.abs(dG).max() < 1e-10
    # range(G) orthogonal to U: loss k
    Gp = rng.standard_normal((25, 4))
    Gp -= U @ (U.T @ Gp)
    L, _ = SN.projector_loss(Gp, U, 0.0)
    assert np.isclose(L, 3.0, rtol=1e-12)
    # invariance under G -> G T (mu = 0)
    G = rng.standard_normal((25, 5))
    T = rng.standard_normal((5, 5)) + 3 * np.eye(5)
    assert np.isclose(SN.projector_loss(G, U, 0.0)[0], SN.projector_loss(G @ T, U, 0.0)[0],
                      rtol=1e-10)
    # conditioning term alone: zero at G^T G = n I
    Q, _ = np.linalg.qr(rng.standard_normal((25, 5)))
    L_pen = SN.projector_loss(np.sqrt(25) * Q, U, 1.0)[0] - SN.projector_loss(np.sqrt(25) * Q, U, 0.0)[0]
    assert abs(L_pen) < 1e-12


@pytest.mark.parametrize("mu", [0.0, 0.05])
def test_projector_gradient_central_differences(mu):
    rng = np.random.default_rng(3)
    G = rng.standard_normal((20, 4))
    U, _ = np.linalg.qr(rng.standard_normal((20, 2)))
    _, dG = SN.projector_loss(G, U, mu)
    h = 1e-6
    num = np.zeros_like(G)
    for i in range(G.shape[0]):
        for j in range(G.shape[1]):
            Gp, Gm = G.copy(), G.copy()
            Gp[i, j] += h
            Gm[i, j] -= h
            num[i, j] = (SN.projector_loss(Gp, U, mu)[0] - SN.projector_loss(Gm, U, mu)[0]) / (2 * h)
    assert np.linalg.norm(num - dG) / np.linalg.norm(dG) < 1e-6


@pytest.mark.parametrize("mu", [0.0, 0.01])
def test_network_gradient_central_differences(mu):
    theta, attrs, U = _case(4)
    L, g = SN.loss_and_grad(theta, attrs, U, SHAPE, mu)
    assert np.isclose(L, SN.projector_loss(SN.forward(theta, attrs, SHAPE)[0], U, mu)[0])
    h = 1e-6
    idx = np.random.default_rng(5).choice(theta.size, 60, replace=False)
    num = np.empty(idx.size)
    for q, i in enumerate(idx):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        num[q] = (SN.loss_and_grad(tp, attrs, U, SHAPE, mu)[0]
                  - SN.loss_and_grad(tm, attrs, U, SHAPE, mu)[0]) / (2 * h)
    assert np.linalg.norm(num - g[idx]) / np.linalg.norm(g[idx]) < 1e-6


def test_forward_special_weights():
    theta, attrs, _ = _case(6)
    W1, b1, W2, b2, W3, b3 = SN.unpack(theta.copy(), SHAPE)
    W3[:] = 0.0
    b3[:] = np.arange(5)
    G, (e, h1, h2) = SN.forward(np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3]),
                                attrs, SHAPE)
    assert np.array_equal(G, np.tile(np.arange(5.0), (attrs.shape[0], 1)))
    W1[:] = 0.0
    th = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])
    _, (e, h1, h2) = SN.forward(th, attrs, SHAPE)
    assert np.allclose(h1, np.tanh(b1))


def test_adam_first_steps_closed_form():
    rng = np.random.default_rng(7)
    g = rng.standard_normal(10)
    th0 = rng.standard_normal(10)
    th1, m, v = SN.adam_step(th0, g, np.zeros(10), np.zeros(10), 1, 0.01)
    # bias-corrected moments equal g and g^2 after one step
    assert np.allclose(th1, th0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    th2, _, _ = SN.adam_step(th1, g, m, v, 2, 0.01)
    assert np.allclose(th2, th1 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-14)
