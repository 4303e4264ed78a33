"""CPU references for the learned coarse correction (test infrastructure only).

* ``unit_response``: K(lam, w) = F^M(0) - G(0) for the unit source e^{i w t} over one
  slice [0, dT], with F^M and G the fine and coarse steps of Eq. (1-7) (complex
  arithmetic, float64).  For a source term amp sin(w t + phi) prod_a g_a the
  slice-n difference of the propagators is P amp Im(e^{i(w T_n + phi)} K).
* ``mlp_forward`` / ``mlp_loss_grad``: the 2 -> 64 -> 64 -> 2 tanh network and the
  gradient of the mean of 0.5 |y - t|^2, in float64, parameters laid out as
  W1[64][2], b1[64], W2[64][64], b2[64], W3[2][64], b3[2].
"""
from __future__ import annotations

import numpy as np

from .phi import b_weights

H = 64


def unit_response(lam, omega, dT: float, M: int, fine_nodes, coarse_nodes) -> np.ndarray:
    lam = np.asarray(lam, dtype=np.float64)
    omega = np.asarray(omega, dtype=np.float64)
    dt = dT / M
    E = np.exp(-lam * dt)
    bF = b_weights(-lam * dt, fine_nodes)
    w = np.zeros(np.broadcast(lam, omega).shape, dtype=np.complex128)
    for m in range(M):
        st = sum(bF[i] * np.exp(1j * omega * (m + c) * dt) for i, c in enumerate(fine_nodes))
        w = E * w + dt * st
    bG = b_weights(-lam * dT, coarse_nodes)
    g = dT * sum(bG[i] * np.exp(1j * omega * c * dT) for i, c in enumerate(coarse_nodes))
    return w - g


def features_targets(lam, omega, dT: float, K: np.ndarray):
    """x = (log(lam dT)/6, w dT - 1); t = 4 K (1 + lam dT) / (dT (w dT)^2) as (re, im)."""
    lam = np.asarray(lam, dtype=np.float64)
    wd = np.asarray(omega, dtype=np.float64) * dT
    x = np.stack([np.log(lam * dT) / 6.0, wd - 1.0], axis=-1)
    scale = 4.0 * (1.0 + lam * dT) / (dT * wd * wd)
    t = np.stack([K.real * scale, K.imag * scale], axis=-1)
    return x, t


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + 2 * H].reshape(H, 2); o += 2 * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + 2 * H].reshape(2, H); o += 2 * H
    b3 = p[o:o + 2]; o += 2
    return W1, b1, W2, b2, W3, b3


def mlp_forward(params, x):
    W1, b1, W2, b2, W3, b3 = unpack(params)
    h1 = np.tanh(x @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ W3.T + b3


def mlp_loss_grad(params, x, t):
    """Mean over samples of 0.5 |y - t|^2 and its gradient (same layout as params)."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    n = x.shape[0]
    h1 = np.tanh(x @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    y = h2 @ W3.T + b3
    e = y - t
    loss = 0.5 * np.sum(e * e) / n
    dy = e / n
    dW3 = dy.T @ h2
    db3 = dy.sum(0)
    dz2 = (dy @ W3) * (1 - h2 * h2)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (1 - h1 * h1)
    dW1 = dz1.T @ x
    db1 = dz1.sum(0)
    grad = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return loss, grad
