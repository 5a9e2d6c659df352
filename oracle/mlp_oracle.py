"""FP64 CPU statement of the covariance surrogate: a small MLP mapping
sightline-pair geometry and hyperparameters to the pair covariance.

TEST INFRASTRUCTURE ONLY -- the CUDA library never imports or runs this file.

The paper computes every covariance entry from the sightline integral
(Sect. 3); the surrogate is this project's approximation of that integral,
trained on the quadrature and checked against it.  Network: 5 inputs -> 3 hidden
layers of 64 units with SiLU -> 2 outputs (the prediction y and a log error
estimate e).  Inputs are the scale-free geometry of the pair in units of L0:
    f1 = ln(sqrt(s_i s_j)/L0) / 4          (mean distance),
    f2 = |s_i - s_j| / (3 L0)              (offset along the sightlines),
    f3 = |u_i - u_j| sqrt(s_i s_j) / (3 L0) (transverse offset),
    f4 = sigma2,   f5 = ln(L0 / 20 pc)
and the target is y = ln K (K = log1p(R), before the taper).  The loss is
    mean (y_pred - y)^2 + lambda * mean rho_q(ln(|y_pred - y| + 1e-5) - e_pred)
with rho_q(u) = u (q - [u < 0]) the pinball (quantile) loss at q = 0.95, so
that e_pred estimates an upper quantile of the log error (Koenker & Bassett
1978), and no gradient flowing from the second term into y_pred.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 5, 64, 2
LAYERS = [(N_IN, N_HID), (N_HID, N_HID), (N_HID, N_HID), (N_HID, N_OUT)]
ERR_FLOOR = 1e-5
ERR_QUANTILE = 0.95


def features(si, sj, chord, sigma2, L0):
    """Scale-free pair features (see module docstring), shape (P, 5)."""
    si, sj = np.asarray(si, float), np.asarray(sj, float)
    L0a = np.broadcast_to(np.asarray(L0, float), si.shape)
    gm = np.sqrt(si * sj) / L0a
    return np.stack([np.log(gm) / 4, np.abs(si - sj) / (3 * L0a),
                     np.asarray(chord, float) * gm / 3,
                     np.broadcast_to(np.asarray(sigma2, float), si.shape),
                     np.log(L0a / 20.0)], axis=1)


def init_params(seed=0):
    """He-style initial weights W (fan_in x fan_out), zero biases."""
    rng = np.random.default_rng(seed)
    return [(rng.standard_normal((i, o)) * np.sqrt(2.0 / i), np.zeros(o)) for i, o in LAYERS]


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, X):
    """Returns (outputs (P, 2), cache of pre-activations and inputs)."""
    h = X
    cache = []
    for k, (W, b) in enumerate(params):
        z = h @ W + b
        cache.append((h, z))
        h = silu(z) if k < len(params) - 1 else z
    return h, cache


def loss_and_grads(params, X, y, lam=0.1, err_target=None):
    """Loss of the module docstring and its gradients (backpropagation).

    The error head's target ln(|y_pred - y| + floor) is held fixed (no
    gradient through it); pass `err_target` to fix it explicitly."""
    out, cache = forward(params, X)
    P = X.shape[0]
    yp, ep = out[:, 0], out[:, 1]
    r = yp - y
    et = np.log(np.abs(r) + ERR_FLOOR) if err_target is None else err_target
    u = et - ep                                   # > 0: error under-estimated
    wq = np.where(u > 0, ERR_QUANTILE, ERR_QUANTILE - 1.0)
    loss = np.mean(r * r) + lam * np.mean(u * wq)
    g_out = np.stack([2.0 * r / P, -lam * wq / P], axis=1)
    grads = [None] * len(params)
    g = g_out
    for k in range(len(params) - 1, -1, -1):
        h, z = cache[k]
        W, _ = params[k]
        if k < len(params) - 1:
            g = g * dsilu(z)
        grads[k] = (h.T @ g, g.sum(axis=0))
        g = g @ W.T
    return loss, grads


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) in place; state = (t, m, v)."""
    t, m, v = state
    t += 1
    newp = []
    for k, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        out = []
        for j, (p, g) in enumerate(((W, gW), (b, gb))):
            m[k][j] = b1 * m[k][j] + (1 - b1) * g
            v[k][j] = b2 * v[k][j] + (1 - b2) * g * g
            mh = m[k][j] / (1 - b1 ** t)
            vh = v[k][j] / (1 - b2 ** t)
            out.append(p - lr * mh / (np.sqrt(vh) + eps))
        newp.append(tuple(out))
    return newp, (t, m, v)


def adam_init(params):
    return (0, [[np.zeros_like(W), np.zeros_like(b)] for W, b in params],
            [[np.zeros_like(W), np.zeros_like(b)] for W, b in params])
