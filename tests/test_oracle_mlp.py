"""Pins for the surrogate-network oracle (CPU): its analytic gradient against
central finite differences of its own loss, and its GELU against the
textbook definition through scipy's normal CDF."""
import numpy as np
import scipy.stats

from oracle import mlp


def test_gelu_is_x_times_normal_cdf():
    z = np.linspace(-6, 6, 1001)
    np.testing.assert_allclose(mlp.gelu(z), z * scipy.stats.norm.cdf(z), rtol=1e-12, atol=1e-14)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), rtol=1e-6, atol=1e-8)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    theta = mlp.init(3) * 0.5
    B = 6
    feats = rng.uniform(-1, 1, size=(B, 4))
    t = rng.random((B, 128))
    t /= t.sum(axis=1, keepdims=True)
    loss, g = mlp.loss_and_grad(theta, feats, t)
    assert g.shape == (mlp.N_PARAMS,)
    idx = rng.choice(mlp.N_PARAMS, size=60, replace=False)
    # parameters inside each block, including every bias block
    offs, at = [], 0
    for name, shape in mlp.SHAPES:
        n = int(np.prod(shape))
        if name == "W1":
            offs += [at + r * 16 + c for r in (0, 7, 200) for c in range(4)]
        else:
            offs += [at, at + n // 2, at + n - 1]
        at += n
    idx = np.concatenate([idx, offs])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, feats, t)[0] - mlp.loss_and_grad(tm, feats, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (i, fd, g[i])


def test_padding_columns_have_zero_gradient():
    rng = np.random.default_rng(2)
    theta = mlp.init(4)
    feats = rng.uniform(-1, 1, size=(5, 4))
    t = np.full((5, 128), 1.0 / 128)
    _, g = mlp.loss_and_grad(theta, feats, t)
    W1 = mlp.unflatten(g)["W1"]
    assert np.all(W1[:, 4:] == 0.0)


def test_loss_is_cross_entropy_of_softmax():
    rng = np.random.default_rng(5)
    theta = mlp.init(6)
    feats = rng.uniform(-1, 1, size=(4, 4))
    t = rng.random((4, 128))
    t /= t.sum(axis=1, keepdims=True)
    q, _ = mlp.forward(theta, feats)
    np.testing.assert_allclose(q.sum(axis=1), 1.0, rtol=1e-12)
    loss, _ = mlp.loss_and_grad(theta, feats, t)
    assert abs(loss - float(-(t * np.log(q)).sum() / 4)) < 1e-12
