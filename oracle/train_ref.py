"""Plain definitions of the training objective and optimiser updates
(Sec. 3.3).  TEST INFRASTRUCTURE ONLY: used by the test suite to check the
GPU training-step kernels; shares nothing with them.

Objective (Sec. 3.3, Eq. 8), per view image I_hat [H, W, 3] and target I:
    L = sum (I - I_hat)^2 + lam * TV(I_hat),
    TV(X) = sum |X[y, x+1] - X[y, x]| + sum |X[y+1, x] - X[y, x]|
(anisotropic: l1 norm of forward differences, per channel, no wrap-around).
The derivative of |d| is taken as sign(d) with sign(0) = 0.

Optimiser (Sec. 3.3: per-group learning rates, 3e-3 for the SH
coefficients and 8e-4 for the positions, decayed by 0.93 per epoch):
    SGD:  p <- p - lr g
    Adam: m <- b1 m + (1 - b1) g ; v <- b2 v + (1 - b2) g^2 ;
          p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)

Parity status: pinned by tests/test_oracle_train.py (TV of constant and ramp
images in closed form, loss gradient by central differences, the first Adam
step equal to lr * sign(g), SGD/Adam convergence on a quadratic).
"""
from __future__ import annotations

import numpy as np


def loss_and_grad(pred, target, lam=0.01, kind="l2"):
    """pred, target: [H, W, 3] (one view).  Returns (loss, dL/dpred)."""
    P = np.asarray(pred, np.float64)
    T = np.asarray(target, np.float64)
    d = P - T
    if kind == "l2":
        loss = float((d * d).sum())
        grad = 2.0 * d
    else:
        loss = float(np.abs(d).sum())
        grad = np.sign(d)
    if lam:
        dx = P[:, 1:, :] - P[:, :-1, :]
        dy = P[1:, :, :] - P[:-1, :, :]
        loss += lam * float(np.abs(dx).sum() + np.abs(dy).sum())
        sx, sy = np.sign(dx), np.sign(dy)
        g = np.zeros_like(P)
        g[:, 1:, :] += sx
        g[:, :-1, :] -= sx
        g[1:, :, :] += sy
        g[:-1, :, :] -= sy
        grad = grad + lam * g
    return loss, grad


def batch_loss_and_grad(pred_packed, target_packed, sizes, lam=0.01, kind="l2"):
    """Packed views ([sum H W, 3]) with sizes [(W, H), ...]."""
    loss, grads, off = 0.0, [], 0
    for (W, H) in sizes:
        n = W * H
        l, g = loss_and_grad(pred_packed[off:off + n].reshape(H, W, 3),
                             target_packed[off:off + n].reshape(H, W, 3), lam, kind)
        loss += l
        grads.append(g.reshape(n, 3))
        off += n
    return loss, np.concatenate(grads)


def sgd_step(p, g, lr):
    return np.asarray(p, np.float64) - lr * np.asarray(g, np.float64)


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step at step number t (1-based); returns (p, m, v)."""
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def lr_at_epoch(lr0, epoch, decay=0.93):
    return lr0 * decay ** epoch
