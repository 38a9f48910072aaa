"""Pins for the oracle's tile-cost network (32 -> 64 ReLU -> 1) and Adam step.

The network has no counterpart in the paper; these tests fix the FP64
reference that the GPU training kernels are checked against: central finite
differences of the loss, a one-unit network worked out by hand, and Adam's
update written out for a single parameter.
"""
import math

import numpy as np
import pytest

import oracle

NIN, NH = 32, 64


def unpack(theta):
    W1 = theta[:NH * NIN].reshape(NH, NIN)
    b1 = theta[NH * NIN:NH * NIN + NH]
    w2 = theta[NH * NIN + NH:NH * NIN + 2 * NH]
    b2 = theta[-1]
    return W1, b1, w2, b2


def test_parameter_count():
    assert oracle.mlp_nparam() == NH * NIN + NH + NH + 1


def test_one_active_unit_by_hand():
    theta = np.zeros(oracle.mlp_nparam())
    W1, b1, w2, _ = unpack(theta)
    W1[3, 0], W1[3, 5], b1[3], w2[3] = 2.0, -1.0, 0.5, 3.0
    theta[-1] = -0.25
    x = np.zeros((2, NIN))
    x[0, 0], x[0, 5] = 1.0, 0.5          # z = 2 - 0.5 + 0.5 = 2 -> y = 6 - 0.25
    x[1, 0], x[1, 5] = 0.0, 4.0          # z = -4 + 0.5 < 0 -> y = -0.25
    y = oracle.mlp_forward(theta, x)
    np.testing.assert_allclose(y, [5.75, -0.25], rtol=0, atol=1e-15)
    loss, g = oracle.mlp_loss_grad(theta, x, np.array([5.0, 0.0]))
    # L = ((0.75)^2 + (0.25)^2) / 2; dL/dy = (0.75, -0.25)
    assert loss == pytest.approx((0.75 ** 2 + 0.25 ** 2) / 2, rel=1e-15)
    gW1, gb1, gw2, gb2 = unpack(g)
    assert gb2 == pytest.approx(0.5, rel=1e-15)
    assert gw2[3] == pytest.approx(0.75 * 2.0, rel=1e-15)
    assert gb1[3] == pytest.approx(0.75 * 3.0, rel=1e-15)
    assert gW1[3, 0] == pytest.approx(0.75 * 3.0 * 1.0, rel=1e-15)
    assert gW1[3, 5] == pytest.approx(0.75 * 3.0 * 0.5, rel=1e-15)
    assert np.count_nonzero(gW1) == 2 and np.count_nonzero(gw2) == 1


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = rng.normal(0, 0.3, oracle.mlp_nparam())
    x = rng.normal(0, 1, (40, NIN))
    t = rng.normal(0, 1, 40)
    loss, g = oracle.mlp_loss_grad(theta, x, t)
    idx = rng.choice(theta.size, 60, replace=False)
    for k in idx:
        e = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[k] += e
        tm[k] -= e
        num = (oracle.mlp_loss_grad(tp, x, t)[0] - oracle.mlp_loss_grad(tm, x, t)[0]) / (2 * e)
        assert num == pytest.approx(g[k], rel=1e-5, abs=1e-8)
    y = oracle.mlp_forward(theta, x)
    assert loss == pytest.approx(np.mean((y - t) ** 2), rel=1e-13)


def test_adam_step_written_out():
    theta = np.array([1.0, -2.0])
    m = np.zeros(2)
    v = np.zeros(2)
    g = np.array([0.5, -4.0])
    oracle.adam_step(theta, g, m, v, t=1, lr=0.1)
    # first step: m_hat = g, v_hat = g^2 -> theta -= lr * sign(g) (up to eps)
    np.testing.assert_allclose(theta, [1.0 - 0.1 * 0.5 / (0.5 + 1e-8), -2.0 + 0.1 * 4 / (4 + 1e-8)],
                               rtol=1e-14)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)
    g2 = np.array([1.0, 1.0])
    oracle.adam_step(theta, g2, m, v, t=2, lr=0.1)
    m2 = 0.9 * 0.1 * g + 0.1 * g2
    v2 = 0.999 * 0.001 * g * g + 0.001 * g2 * g2
    step = 0.1 * (m2 / (1 - 0.81)) / (np.sqrt(v2 / (1 - 0.999 ** 2)) + 1e-8)
    np.testing.assert_allclose(theta, np.array([1.0 - 0.1 * 0.5 / (0.5 + 1e-8),
                                                -2.0 + 0.1 * 4 / (4 + 1e-8)]) - step, rtol=1e-12)


def test_training_lowers_the_loss():
    rng = np.random.default_rng(1)
    x = rng.random((256, NIN))
    t = 2.0 * x[:, 0] + np.sin(3 * x[:, 1]) + x[:, 16] ** 2
    theta = rng.normal(0, 1.0 / math.sqrt(NIN), oracle.mlp_nparam())
    theta[NH * NIN:NH * NIN + NH] = 0.0
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    first = oracle.mlp_loss_grad(theta, x, t)[0]
    for step in range(1, 301):
        loss, g = oracle.mlp_loss_grad(theta, x, t)
        oracle.adam_step(theta, g, m, v, step, lr=3e-3)
    assert loss < 0.05 * first
