"""Pins for the training-objective and optimiser definitions (Sec. 3.3)."""
import numpy as np

from oracle import train_ref as TR


def test_tv_of_constant_and_ramp_images():
    c = np.full((7, 9, 3), 0.3)
    loss, g = TR.loss_and_grad(c, c, lam=1.0)
    assert loss == 0.0 and np.all(g == 0)
    # horizontal ramp a*x: every x-difference is a, y-differences vanish
    a = 0.25
    ramp = np.broadcast_to(a * np.arange(9.0)[None, :, None], (7, 9, 3)).copy()
    loss, _ = TR.loss_and_grad(ramp, ramp, lam=1.0)
    assert abs(loss - a * 8 * 7 * 3) < 1e-12
    # vertical ramp: the same with the roles swapped
    vr = np.broadcast_to(a * np.arange(7.0)[:, None, None], (7, 9, 3)).copy()
    loss, _ = TR.loss_and_grad(vr, vr, lam=1.0)
    assert abs(loss - a * 6 * 9 * 3) < 1e-12


def test_data_term_is_sum_of_squares_and_abs():
    rng = np.random.default_rng(0)
    p, t = rng.normal(size=(5, 4, 3)), rng.normal(size=(5, 4, 3))
    l2, _ = TR.loss_and_grad(p, t, lam=0.0)
    l1, g1 = TR.loss_and_grad(p, t, lam=0.0, kind="l1")
    assert abs(l2 - ((p - t) ** 2).sum()) < 1e-12 and abs(l1 - np.abs(p - t).sum()) < 1e-12
    assert np.array_equal(g1, np.sign(p - t))


def test_loss_gradient_by_central_differences():
    rng = np.random.default_rng(1)
    p, t = rng.normal(size=(6, 5, 3)), rng.normal(size=(6, 5, 3))
    loss, g = TR.loss_and_grad(p, t, lam=0.37)
    h = 1e-7  # differences between neighbours are O(1): no kink within h
    num = np.zeros_like(p)
    for idx in np.ndindex(p.shape):
        q = p.copy()
        q[idx] += h
        lp, _ = TR.loss_and_grad(q, t, lam=0.37)
        q[idx] -= 2 * h
        lm, _ = TR.loss_and_grad(q, t, lam=0.37)
        num[idx] = (lp - lm) / (2 * h)
    assert np.abs(num - g).max() < 1e-5


def test_first_adam_step_is_lr_times_sign():
    rng = np.random.default_rng(2)
    p, g = rng.normal(size=50), rng.normal(size=50)
    p1, m, v = TR.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr=3e-3, eps=0.0)
    assert np.allclose(p1, p - 3e-3 * np.sign(g), atol=1e-15)


def test_optimisers_descend_a_quadratic():
    x = np.array([3.0, -2.0, 0.5])
    p, m, v = x.copy(), np.zeros(3), np.zeros(3)
    for t in range(1, 3001):
        p, m, v = TR.adam_step(p, 2 * p, m, v, t, lr=1e-2)
    assert np.abs(p).max() < 1e-2
    q = x.copy()
    for _ in range(200):
        q = TR.sgd_step(q, 2 * q, 0.1)
    assert np.abs(q).max() < 1e-12


def test_learning_rate_schedule():
    assert abs(TR.lr_at_epoch(3e-3, 0) - 3e-3) < 1e-18
    assert abs(TR.lr_at_epoch(8e-4, 20) - 8e-4 * 0.93 ** 20) < 1e-18
