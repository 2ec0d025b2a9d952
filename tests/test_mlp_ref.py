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


def _torch_net(p, n_in, H, n_out):
    # the flat layout written out independently of mlp_ref.unpack:
    # [W1 (H x n_in) | b1 (H) | W2 (H x H) | b2 (H) | W3 (n_out x H) | b3 (n_out)], row-major
    import torch
    q = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    o1 = H * n_in
    o2 = o1 + H
    o3 = o2 + H * H
    o4 = o3 + H
    o5 = o4 + n_out * H
    W1, b1 = q[:o1].view(H, n_in), q[o1:o2]
    W2, b2 = q[o2:o3].view(H, H), q[o3:o4]
    W3, b3 = q[o4:o5].view(n_out, H), q[o5:]
    assert b3.numel() == n_out
    return q, (W1, b1, W2, b2, W3, b3)


@pytest.mark.parametrize("seed", range(4))
def test_forward_loss_and_gradient_match_torch_autograd(seed):
    torch = pytest.importorskip("torch")
    import torch.nn.functional as F
    p, x, t, mask, n_in, H, n_out = _setup(100 + seed, n_in=6, H=9, n_out=5, rows=7)
    q, (W1, b1, W2, b2, W3, b3) = _torch_net(p, n_in, H, n_out)
    X = torch.tensor(x, dtype=torch.float64)
    y = F.linear(F.relu(F.linear(F.relu(F.linear(X, W1, b1)), W2, b2)), W3, b3)
    Mk = torch.tensor(mask, dtype=torch.float64)
    L = (Mk * (y - torch.tensor(t, dtype=torch.float64)) ** 2).sum() / Mk.sum()
    L.backward()
    yr, _ = M.forward(p, x, n_in, H, n_out)
    np.testing.assert_allclose(yr, y.detach().numpy(), rtol=1e-12, atol=1e-12)
    assert M.loss(p, x, t, mask, n_in, H, n_out) == pytest.approx(L.item(), rel=1e-12)
    np.testing.assert_allclose(M.grad(p, x, t, mask, n_in, H, n_out), q.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_adam_matches_torch_optimizer_over_several_steps():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    p = rng.normal(size=30)
    w = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([w], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    m1 = np.zeros(30)
    m2 = np.zeros(30)
    for step in range(1, 8):
        g = rng.normal(size=30) * (1 + step)
        w.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        q, m1, m2 = M.adam_step(p, g, m1, m2, step, 3e-3)
        np.testing.assert_allclose(q - p, w.detach().numpy() - p, rtol=1e-9, atol=1e-15)
        p = w.detach().numpy().copy()
