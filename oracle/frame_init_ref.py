"""Plain definition of the video frame initialisation (Sec. 3.4, "Video
Synthesis").  TEST INFRASTRUCTURE ONLY: used by the test suite to check
the GPU kernels; shares no code with them.

Given the trained cloud S1 of one frame (positions x_i with SH, opacity,
radius) and an initial cloud S2 for the next frame (positions y_j), the
paper
  1. moves the positions of S2 by gradient descent (Adam) on the Chamfer
     distance (the equation of Sec. 3.4)
        CD(S1, S2) = 1/|S1| sum_i min_j |x_i - y_j|^2
                   + 1/|S2| sum_j min_i |x_i - y_j|^2 ;
  2. gives each refined y_j the mean parameters of its k closest points
     of S1.

Readings where the paper leaves details open (each implemented below):
  F1 nearest points: by fp32 squared distance ((dx dx + dy dy) + dz dz),
     ties by lower index (the same neighbour search as the coarse-to-fine
     update); the distance values entering CD are taken in fp64 from the
     fp32 positions.
  F2 gradient: with the nearest points held fixed (the minimum is
     piecewise smooth),
        dCD/dy_j = 2/|S1| sum_{i: nn(x_i) = j} (y_j - x_i)
                 + 2/|S2| (y_j - x_nn(y_j)).
  F3 optimiser: Adam (0.9, 0.999, 1e-8) on the positions of S2 only, with
     a constant learning rate (default 1e-3) for a fixed number of steps
     (default 100); positions are stored in fp32 after every step.
  F4 parameters: the plain mean of the SH coefficients, opacity and radius
     of the k closest points of S1 (default k = 4), by the same neighbour
     search; fp64 means.
  The loss history holds CD before every step and after the last one.

Parity status: pinned by tests/test_oracle_frame_init.py (CD and its
gradient for identical clouds, single points and small translations in
closed form; CD against scipy's k-d tree; the gradient by central
differences; parameter means on a lattice; descent of the loop).
"""
from __future__ import annotations

import numpy as np

from oracle import refine_ref as RR
from oracle import train_ref as TR

F32 = np.float32


def nearest(q, ref):
    """F1: index of the nearest point of ref for every point of q."""
    idx, _ = RR.knn(np.asarray(q, F32), 1, ref=np.asarray(ref, F32))
    return idx[:, 0]


def chamfer(p1, p2):
    """CD(S1, S2) (fp64), dCD/dp2 (fp64) and the two nearest-point maps."""
    x = np.asarray(p1, F32)
    y = np.asarray(p2, F32)
    nn12 = nearest(x, y)  # for every x_i its nearest y
    nn21 = nearest(y, x)  # for every y_j its nearest x
    x64, y64 = x.astype(np.float64), y.astype(np.float64)
    d12 = y64[nn12] - x64
    d21 = y64 - x64[nn21]
    cd = (d12 * d12).sum() / len(x) + (d21 * d21).sum() / len(y)
    grad = 2.0 / len(y) * d21
    np.add.at(grad, nn12, 2.0 / len(x) * d12)
    return float(cd), grad, nn12, nn21


def mean_params(p2, p1, attrs1, k):
    """F4: means of the k closest points' parameters, and their indices."""
    idx, _ = RR.knn(np.asarray(p2, F32), k, ref=np.asarray(p1, F32))
    return [np.asarray(a, np.float64)[idx].mean(axis=1) for a in attrs1], idx


def frame_init(p1, attrs1, p2, iters=100, lr=1e-3, k=4, b1=0.9, b2=0.999, eps=1e-8):
    """Steps 1-2.  attrs1: [sh, opacity, radius] of S1.  Returns (positions
    of S2 after the descent (fp32), [sh, opacity, radius] of S2 (fp64),
    loss history (iters + 1 values))."""
    y = np.asarray(p2, F32).copy()
    m = np.zeros(y.shape)
    v = np.zeros(y.shape)
    hist = []
    for t in range(1, iters + 1):
        cd, g, _, _ = chamfer(p1, y)
        hist.append(cd)
        y64, m, v = TR.adam_step(y, g, m, v, t, lr, b1, b2, eps)
        y = y64.astype(F32)
    hist.append(chamfer(p1, y)[0])
    params, _ = mean_params(y, p1, attrs1, k)
    return y, params, hist
