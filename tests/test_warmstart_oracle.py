"""Pins of the numpy reference of the learned initial-guess network (oracle/warmstart_oracle.py)
against things other than itself: a library correlation, adjoint identities, closed forms and
finite differences of its own forward map."""
import numpy as np
import pytest

import synthetic
from oracle import warmstart_oracle as wo


def _r(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_conv_matches_scipy_correlate():
    signal = pytest.importorskip("scipy.signal")
    x = _r((5, 6, 7, 3), 1)
    W = _r((27, 3, 2), 2)
    y = wo.conv(x, W)
    for co in range(2):
        ref = np.zeros((5, 6, 7))
        for ci in range(3):
            k = W[:, ci, co].reshape(3, 3, 3)  # taps ordered (dz, dy, dx), each -1..1
            ref += signal.correlate(x[..., ci], k, mode="same")
        assert np.max(np.abs(y[..., co] - ref)) < 1e-12


def test_conv_adjoints():
    x = _r((4, 5, 6, 3), 3)
    W = _r((27, 3, 4), 4)
    g = _r((4, 5, 6, 4), 5)
    lhs = np.sum(wo.conv(x, W) * g)
    assert abs(lhs - np.sum(x * wo.conv_bwd_data(g, W))) < 1e-10 * abs(lhs)
    assert abs(lhs - np.sum(W * wo.conv_bwd_weight(x, g))) < 1e-10 * abs(lhs)


def test_identity_tap_is_identity():
    x = _r((3, 4, 5, 2), 6)
    W = np.zeros((27, 2, 2))
    W[13] = np.eye(2)  # centre tap (0, 0, 0)
    assert np.array_equal(wo.conv(x, W), x)
    W = np.zeros((27, 2, 2))
    W[14] = np.eye(2)  # tap (0, 0, +1): y[x] = x[x + 1], zero at the far end
    y = wo.conv(x, W)
    assert np.array_equal(y[:, :, :-1], x[:, :, 1:]) and np.all(y[:, :, -1] == 0)


def test_pool_up_relations():
    x = _r((2, 3, 4, 2), 7)
    g = _r((4, 6, 8, 2), 8)
    assert np.allclose(wo.pool(wo.up(x)), x)
    assert abs(np.sum(wo.up(x) * g) - np.sum(x * wo.up_T(g))) < 1e-12
    assert abs(np.sum(wo.pool(g) * x) - np.sum(g * wo.pool_T(x))) < 1e-12


def test_faces_cells_maps():
    n = 6
    m = (n + 1) * n * n * 3 + n ** 3
    P = _r((n, n, n, 4), 9)
    y = _r(m, 10)
    assert abs(np.sum(wo.faces(P, n) * y) - np.sum(P * wo.faces_T(y, n))) < 1e-10
    # constant cell field: interior faces take the constant, wall faces 0
    u, v, w, p = wo._split(wo.faces(np.ones((n, n, n, 4)), n), n)
    assert np.all(u[:, :, 1:-1] == 1) and np.all(u[:, :, [0, -1]] == 0)
    assert np.all(v[:, 1:-1] == 1) and np.all(w[1:-1] == 1) and np.all(p == 1)
    # a linear face field x -> its cell means are the values at the cell centres
    b = np.zeros(m)
    u, v, w, p = wo._split(b, n)
    u[...] = np.arange(n + 1)[None, None, :]
    c = wo.cells(b, n)
    assert np.allclose(c[..., 0], np.arange(n)[None, None, :] + 0.5)


def _problem(n, seed):
    m = (n + 1) * n * n * 3 + n ** 3
    b = _r(m, seed)
    xs = _r(m, seed + 1)
    return b, xs


def test_forward_positively_homogeneous():
    n = 8
    w = synthetic.net_weights(0)
    b, _ = _problem(n, 11)
    x1 = wo.predict(b, w, n, 0.3)
    x2 = wo.predict(2.5 * b, w, n, 0.3)
    assert np.max(np.abs(x2 - 2.5 * x1)) < 1e-12 * np.max(np.abs(x2))


def test_gradient_matches_finite_differences():
    n = 16  # level 3 is 2^3, so every tap of the coarsest convolutions is exercised
    w = synthetic.net_weights(1) * 0.5
    b, xs = _problem(n, 12)
    L, g = wo.loss_and_grad(b, xs, w, n, 0.7)
    assert abs(L - wo.loss(b, xs, w, n, 0.7)) < 1e-14 * L
    rng = np.random.default_rng(13)
    # one random coordinate in every weight tensor, plus a random direction
    offs = np.cumsum([0] + [a * b_ * c for a, b_, c in wo.SHAPES])
    coords = [int(rng.integers(offs[i], offs[i + 1])) for i in range(len(wo.SHAPES))]
    eps = 1e-6
    for q in coords:
        e = np.zeros_like(w)
        e[q] = eps
        fd = (wo.loss(b, xs, w + e, n, 0.7) - wo.loss(b, xs, w - e, n, 0.7)) / (2 * eps)
        # central differences: truncation ~eps^2, cancellation ~1e-16 L / eps ~ 1e-10
        assert abs(fd - g[q]) <= 1e-4 * abs(g[q]) + 1e-9, (q, fd, g[q])
    d = rng.standard_normal(w.size)
    d /= np.linalg.norm(d)
    fd = (wo.loss(b, xs, w + eps * d, n, 0.7) - wo.loss(b, xs, w - eps * d, n, 0.7)) / (2 * eps)
    assert abs(fd - g @ d) <= 1e-6 * np.linalg.norm(g)


def test_adam_first_step_moves_by_learning_rate():
    # Adam's bias-corrected first step is lr * g / (|g| + eps) per coordinate
    w = _r(50, 14)
    g = _r(50, 15)
    w1 = wo.adam(w.copy(), g, np.zeros(50), np.zeros(50), 1, 1e-2, eps=0.0)
    assert np.allclose(w - w1, 1e-2 * np.sign(g))


def test_residual_form_gradient_matches_finite_differences():
    import oracle
    n = 16
    o = oracle.Oracle(n, coarsest_max=8)
    act, _ = o.masks()
    w = synthetic.net_weights(2) * 0.5
    b, xs = _problem(n, 20)
    b[~act] = 0.0
    xs[~act] = 0.0
    L, g = wo.loss_and_grad(b, xs, w, n, 0.7, apply=o.apply)
    assert abs(L - wo.loss(b, xs, w, n, 0.7, apply=o.apply)) < 1e-13 * L
    rng = np.random.default_rng(21)
    d = rng.standard_normal(w.size)
    d /= np.linalg.norm(d)
    eps = 1e-6
    fd = (wo.loss(b, xs, w + eps * d, n, 0.7, apply=o.apply) - wo.loss(b, xs, w - eps * d, n, 0.7, apply=o.apply)) / (2 * eps)
    assert abs(fd - g @ d) <= 1e-5 * np.linalg.norm(g)
