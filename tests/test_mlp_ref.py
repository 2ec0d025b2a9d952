"""Pins for the numpy restatement of the scheduler network (no GPU)."""
import numpy as np
import pytest

from oracle import mlp_ref as M


def _setup(seed, n_in=5, H=7, n_out=4, rows=6):
    rng = np.random.default_rng(seed)
    npar = H * n_in + H + H * H + H + n_out * H + n_out
    p = rng.normal(0, 0.5, npar)
    x = rng.normal(0, 1, (rows, n_in))
    t = rng.normal(0, 1, (rows, n_out))
    mask = (rng.random((rows, n_out)) < 0.7).astype(float)
    mask[0, 0] = 1.0
    return p, x, t, mask, n_in, H, n_out


@pytest.mark.parametrize("seed", range(6))
def test_gradient_matches_central_differences(seed):
    p, x, t, mask, n_in, H, n_out = _setup(seed)
    g = M.grad(p, x, t, mask, n_in, H, n_out)
    eps = 1e-6
    num = np.zeros_like(p)
    for i in range(p.size):
        q = p.copy(); q[i] += eps
        r = p.copy(); r[i] -= eps
        num[i] = (M.loss(q, x, t, mask, n_in, H, n_out) - M.loss(r, x, t, mask, n_in, H, n_out)) / (2 * eps)
    # relu kinks are measure-zero for random inputs
    np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-7)


def test_forward_matches_explicit_loops():
    p, x, t, mask, n_in, H, n_out = _setup(11, rows=3)
    W1, b1, W2, b2, W3, b3 = M.unpack(p, n_in, H, n_out)
    y, _ = M.forward(p, x, n_in, H, n_out)
    for r in range(3):
        h1 = [max(0.0, sum(W1[j, i] * x[r, i] for i in range(n_in)) + b1[j]) for j in range(H)]
        h2 = [max(0.0, sum(W2[j, k] * h1[k] for k in range(H)) + b2[j]) for j in range(H)]
        for o in range(n_out):
            assert y[r, o] == pytest.approx(sum(W3[o, k] * h2[k] for k in range(H)) + b3[o], rel=1e-12)


def test_adam_first_step_is_lr_times_sign():
    # with bias correction, the first Adam step moves every parameter by ~lr against its gradient sign
    rng = np.random.default_rng(3)
    p = rng.normal(size=20)
    g = rng.normal(size=20)
    q, m1, m2 = M.adam_step(p, g, np.zeros(20), np.zeros(20), 1, 0.01)
    np.testing.assert_allclose(q - p, -0.01 * np.sign(g), rtol=1e-6)


def test_training_by_gradient_descent_fits_a_linear_target():
    rng = np.random.default_rng(5)
    n_in, H, n_out = 3, 16, 2
    npar = H * n_in + H + H * H + H + n_out * H + n_out
    p = rng.normal(0, 0.3, npar)
    x = rng.normal(size=(64, n_in))
    t = np.stack([x[:, 0] - 2 * x[:, 1], 0.5 * x[:, 2] + 1], axis=1)
    mask = np.ones_like(t)
    l0 = M.loss(p, x, t, mask, n_in, H, n_out)
    m1 = np.zeros(npar); m2 = np.zeros(npar)
    for s in range(1, 801):
        p, m1, m2 = M.adam_step(p, M.grad(p, x, t, mask, n_in, H, n_out), m1, m2, s, 1e-2)
    assert M.loss(p, x, t, mask, n_in, H, n_out) < 0.05 * l0
