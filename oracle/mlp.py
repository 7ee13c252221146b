"""FP64 statement of the q/sketch-size selector network and its features.

TEST INFRASTRUCTURE ONLY: imported by tests and by the training script's
checks; never by the product path.

The selector is a multilayer perceptron with three hidden layers of 64 ReLU
units.  Its parameters are one packed vector, layer by layer: W_l (out x in,
row-major) followed by b_l.  Loss: masked mean squared error.  Optimiser:
Adam (Kingma & Ba, 2015) with bias correction.

Features of the q = 0 sketch (Algorithm 1 with q = 0: Y0 = A S Omega), from
the singular values s_1 >= ... >= s_r2 of Y0 (eigenvalues of Y0^T Y0):
  f0 = log10(s_{i4} / s_1), i4 = max(1, r2 // 4)
  f1 = log10(s_{i2} / s_1), i2 = max(1, r2 // 2)
  f2 = log10(s_{r2} / s_1)
  f3 = log10(r2 s_{r2}^2 / sum_i s_i^2)        (flatness of the sketch tail)
  f4 = log10(m) / 4, f5 = log10(n) / 4, f6 = log10(r2) / 3,
  f7 = log2(r1 / r2) / 3                        (probe sketch ratio)
(index s_i counts from 1; singular values below 1e-30 s_1 are clamped.)
"""
import numpy as np

D_IN, HID, D_OUT = 8, 64, 15
LAYERS = [(HID, D_IN), (HID, HID), (HID, HID), (D_OUT, HID)]
N_PARAMS = sum(o * i + o for o, i in LAYERS)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, off = [], 0
    for o, i in LAYERS:
        W = p[off:off + o * i].reshape(o, i)
        off += o * i
        b = p[off:off + o]
        off += o
        out.append((W, b))
    return out


def init_params(seed=0):
    """He-style initialisation (normal, std sqrt(2 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for o, i in LAYERS:
        parts.append(rng.standard_normal(o * i) * np.sqrt(2.0 / i))
        parts.append(np.zeros(o))
    return np.concatenate(parts)


def forward(p, X):
    """Y = W4 relu(W3 relu(W2 relu(W1 x + b1) + b2) + b3) + b4 for each row x of X."""
    X = np.asarray(X, dtype=np.float64)
    acts = [X]
    h = X
    layers = unpack(p)
    for li, (W, b) in enumerate(layers):
        z = h @ W.T + b
        h = np.maximum(z, 0.0) if li < len(layers) - 1 else z
        acts.append(h)
    return h, acts


def loss_grad(p, X, T, M):
    """Masked MSE L = sum M (Y - T)^2 / max(sum M, 1) and dL/dp (packed)."""
    Y, acts = forward(p, X)
    T = np.asarray(T, dtype=np.float64)
    M = np.asarray(M, dtype=np.float64)
    cnt = max(M.sum(), 1.0)
    R = (Y - T) * M
    loss = float((R * (Y - T)).sum() / cnt)
    layers = unpack(p)
    grads = [None] * len(layers)
    delta = 2.0 * R / cnt                      # dL/dY
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        h_in = acts[li]
        grads[li] = (delta.T @ h_in, delta.sum(axis=0))
        if li > 0:
            delta = (delta @ W) * (acts[li] > 0.0)
    flat = []
    for gW, gb in grads:
        flat.append(gW.reshape(-1))
        flat.append(gb)
    return loss, np.concatenate(flat)


def adam(p, m, v, g, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (step counts from 1); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def features_from_sketch(Y0, m, n, r1):
    """The selector's input features from the q = 0 sketch Y0 = A S Omega (m x r2)."""
    Y0 = np.asarray(Y0, dtype=np.float64)
    r2 = Y0.shape[1]
    lam = np.linalg.eigvalsh(Y0.T @ Y0)[::-1]
    s = np.sqrt(np.maximum(lam, 0.0))
    s = np.maximum(s, 1e-30 * s[0])
    i4, i2 = max(1, r2 // 4), max(1, r2 // 2)
    f = [np.log10(s[i4 - 1] / s[0]), np.log10(s[i2 - 1] / s[0]), np.log10(s[-1] / s[0]),
         np.log10(r2 * s[-1] ** 2 / np.sum(s ** 2)),
         np.log10(m) / 4, np.log10(n) / 4, np.log10(r2) / 3, np.log2(r1 / r2) / 3]
    return np.array(f)
