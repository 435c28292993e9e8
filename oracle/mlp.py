"""FP64 reference of the p_det surrogate network (TEST INFRASTRUCTURE ONLY).

A 4-layer perceptron d_in -> w -> w -> w -> 1, ReLU between layers, logit output; loss =
mean binary cross entropy of sigmoid(logit) against labels in {0, 1}; Adam with bias
correction (Kingma & Ba, ICLR 2015).  Parameters are one vector in the order
W1[w][d_in] b1 W2[w][w] b2 W3[w][w] b3 W4[1][w] b4 -- the layout of the CUDA model.
Plain numpy, no batching tricks: every formula is the textbook one.
"""
import numpy as np


def shapes(d, w):
    return [(w, d), (w,), (w, w), (w,), (w, w), (w,), (1, w), (1,)]


def unpack(theta, d, w):
    theta = np.asarray(theta, np.float64)
    out, o = [], 0
    for s in shapes(d, w):
        n = int(np.prod(s))
        out.append(theta[o:o + n].reshape(s))
        o += n
    assert o == theta.size
    return out


def forward(theta, X, d, w):
    """Layer outputs (post-ReLU hidden activations) and logits."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta, d, w)
    X = np.asarray(X, np.float64)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    h3 = np.maximum(h2 @ W3.T + b3, 0.0)
    z = (h3 @ W4.T + b4)[:, 0]
    return (h1, h2, h3), z


def bce(z, y):
    """Mean of -y log s - (1 - y) log(1 - s), s = sigmoid(z), in a cancellation-free form."""
    z = np.asarray(z, np.float64)
    y = np.asarray(y, np.float64)
    return float(np.mean(np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def loss_and_grad(theta, X, y, d, w):
    """Loss and its gradient by back-propagation (chain rule through each layer)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta, d, w)
    X = np.asarray(X, np.float64)
    y = np.asarray(y, np.float64)
    (h1, h2, h3), z = forward(theta, X, d, w)
    B = len(y)
    dz = (1.0 / (1.0 + np.exp(-z)) - y) / B           # d loss / d z
    gW4 = dz[None, :] @ h3
    gb4 = np.array([dz.sum()])
    dh3 = np.outer(dz, W4[0]) * (h3 > 0)
    gW3 = dh3.T @ h2
    gb3 = dh3.sum(0)
    dh2 = (dh3 @ W3) * (h2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ W2) * (h1 > 0)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4)])
    return bce(z, y), g


def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step count t >= 1); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def predict(theta, X, d, w):
    _, z = forward(theta, X, d, w)
    return 1.0 / (1.0 + np.exp(-z))
