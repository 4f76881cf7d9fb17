"""Pins for the warm-start network's oracle: finite differences of the loss, the closed form of
the first AdamW step, the identity start, and the feature layout."""
import numpy as np
import pytest

from oracle import mlp as M


def small_params(rng, widths=(17, 6, 5, 4, 8), scale=0.5):
    return [(scale * rng.standard_normal((o, i)), scale * rng.standard_normal(o)) for i, o in zip(widths[:-1], widths[1:])]


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    params = small_params(rng)
    X = rng.standard_normal((7, 17))
    T = rng.standard_normal((7, 8))
    loss, grads = M.loss_and_grads(params, X, T)
    eps = 1e-6
    for li, (W, b) in enumerate(params):
        for which, arr in ((0, W), (1, b)):
            for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(3)]:
                pp = [(W_.copy(), b_.copy()) for W_, b_ in params]
                pm = [(W_.copy(), b_.copy()) for W_, b_ in params]
                pp[li][which][idx] += eps
                pm[li][which][idx] -= eps
                fd = (M.loss_and_grads(pp, X, T)[0] - M.loss_and_grads(pm, X, T)[0]) / (2 * eps)
                assert grads[li][which][idx] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_zero_last_layer_gives_the_previous_solution():
    rng = np.random.default_rng(1)
    params = small_params(rng)
    W, b = params[-1]
    params[-1] = (np.zeros_like(W), np.zeros_like(b))
    X = rng.standard_normal((5, 17))
    y, _ = M.forward(params, X)
    np.testing.assert_array_equal(X[:, :8] + y, X[:, :8])


def test_first_adamw_step_closed_form():
    """At t = 1 the bias-corrected moments are g and g^2, so the step is
    -lr (g / (|g| + eps) + wd p)."""
    p = [(np.array([[0.5, -2.0]]), np.array([0.25]))]
    g = [(np.array([[3.0, -0.001]]), np.array([0.0]))]
    m = [[np.zeros((1, 2)), np.zeros(1)]]
    v = [[np.zeros((1, 2)), np.zeros(1)]]
    lr, wd, eps = 0.1, 0.01, 1e-8
    out = M.adamw_step(p, g, m, v, 1, lr, eps=eps, wd=wd)
    expW = p[0][0] - lr * (g[0][0] / (np.abs(g[0][0]) + eps) + wd * p[0][0])
    np.testing.assert_allclose(out[0][0], expW, rtol=1e-12)
    np.testing.assert_allclose(out[0][1], p[0][1] - lr * wd * p[0][1], rtol=1e-12)


def test_feature_rows_round_trip():
    rng = np.random.default_rng(2)
    J = rng.standard_normal((3, 2, 4, 2, 2)) + 1j * rng.standard_normal((3, 2, 4, 2, 2))
    BZ = rng.standard_normal(J.shape) + 1j * rng.standard_normal(J.shape)
    X = M.features(J, BZ, [0.0, 0.5, 1.0])
    assert X.shape == (3 * 2 * 4, 17)
    np.testing.assert_array_equal(M.rows_to_jones(X[:, :8], 3, 2, 4), J)
    np.testing.assert_array_equal(M.rows_to_jones(X[:, 8:16], 3, 2, 4), BZ)
    assert X[1 * 2 * 4, 16] == 0.5 and X[2 * 2 * 4, 16] == 1.0
