"""Plain numpy (float64) restatement of the scheduler network -- TEST INFRASTRUCTURE ONLY.

Only tests/ may import this module; the CUDA library never uses it.  It
restates, with the textbook formulas, what the network kernels compute:

    h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  y = W3 h2 + b3
    L  = sum(mask * (y - t)^2) / sum(mask)

the gradient of L by backpropagation, and one Adam step (Kingma & Ba, with
bias correction).  Parameters use the library's flat layout
[W1 (H x n_in) | b1 | W2 (H x H) | b2 | W3 (n_out x H) | b3].
Pinned by central finite differences in tests/test_mlp_ref.py.
"""
import numpy as np


def unpack(p, n_in, H, n_out):
    p = np.asarray(p, np.float64)
    i = 0
    out = []
    for shape in ((H, n_in), (H,), (H, H), (H,), (n_out, H), (n_out,)):
        k = int(np.prod(shape))
        out.append(p[i:i + k].reshape(shape))
        i += k
    assert i == p.size
    return out


def pack(parts):
    return np.concatenate([np.asarray(a, np.float64).ravel() for a in parts])


def forward(p, x, n_in, H, n_out):
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, H, n_out)
    x = np.asarray(x, np.float64).reshape(-1, n_in)
    a1 = x @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ W3.T + b3
    return y, (x, a1, h1, a2, h2)


def loss(p, x, t, mask, n_in, H, n_out):
    y, _ = forward(p, x, n_in, H, n_out)
    m = np.asarray(mask, np.float64).reshape(y.shape)
    d = y - np.asarray(t, np.float64).reshape(y.shape)
    return float((m * d * d).sum() / m.sum())


def grad(p, x, t, mask, n_in, H, n_out):
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, H, n_out)
    y, (x, a1, h1, a2, h2) = forward(p, x, n_in, H, n_out)
    m = np.asarray(mask, np.float64).reshape(y.shape)
    dy = 2.0 * m * (y - np.asarray(t, np.float64).reshape(y.shape)) / m.sum()
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    dh2 = (dy @ W3) * (a2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ W2) * (a1 > 0)
    gW1 = dh1.T @ x
    gb1 = dh1.sum(0)
    return pack([gW1, gb1, gW2, gb2, gW3, gb3])


def adam_step(p, g, m1, m2, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step; step counts from 1.  Returns (p, m1, m2)."""
    m1 = b1 * m1 + (1 - b1) * g
    m2 = b2 * m2 + (1 - b2) * g * g
    mh = m1 / (1 - b1 ** step)
    vh = m2 / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m1, m2
