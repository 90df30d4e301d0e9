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


def _torch_adamw_steps(theta0, grads, lr, wd, beta1=0.9, beta2=0.999, eps=1e-8):
    """The same steps through torch.optim.AdamW (float64, two parameter groups:
    weight matrices with decay, biases without; the W1 padding columns are
    left out of the optimiser)."""
    import torch
    P = {name: torch.tensor(a, dtype=torch.float64, requires_grad=True) for name, a in mlp.unflatten(theta0).items()}
    pad = torch.zeros(256, 16, dtype=torch.bool)
    pad[:, 4:] = True
    W1 = P["W1"]
    W1_act = torch.tensor(mlp.unflatten(theta0)["W1"][:, :4], dtype=torch.float64, requires_grad=True)
    groups = [{"params": [W1_act] + [P[n] for n, _ in mlp.SHAPES if n.startswith("W") and n != "W1"],
               "weight_decay": wd},
              {"params": [P[n] for n, _ in mlp.SHAPES if n.startswith("b")], "weight_decay": 0.0}]
    opt = torch.optim.AdamW(groups, lr=lr, betas=(beta1, beta2), eps=eps)
    for g in grads:
        G = mlp.unflatten(g)
        W1_act.grad = torch.tensor(G["W1"][:, :4])
        for n, _ in mlp.SHAPES:
            if n != "W1":
                P[n].grad = torch.tensor(G[n])
        opt.step()
    out = {n: P[n].detach().numpy().copy() for n, _ in mlp.SHAPES}
    w1 = W1.detach().numpy().copy()
    w1[:, :4] = W1_act.detach().numpy()
    out["W1"] = w1
    return mlp.flatten(out)


def test_adamw_matches_torch_optimizer():
    """Three AdamW steps of the oracle against torch.optim.AdamW (a library
    routine of the same published method) on random gradients."""
    rng = np.random.default_rng(8)
    theta = mlp.init(2)
    grads = [rng.standard_normal(mlp.N_PARAMS) * s for s in (1e-3, 3e-2, 1e-5)]
    for g in grads:
        mlp.unflatten(g)["W1"][:, 4:] = 0.0
    lr, wd = 2e-3, 0.05
    th, m, v = theta.copy(), np.zeros(mlp.N_PARAMS), np.zeros(mlp.N_PARAMS)
    for t, g in enumerate(grads, start=1):
        th, m, v = mlp.adamw_step(th, g, m, v, t, lr, wd)
    ref = _torch_adamw_steps(theta, grads, lr, wd)
    np.testing.assert_allclose(th, ref, rtol=1e-13, atol=1e-15)
    # the padding columns never move, whatever their gradient
    g = rng.standard_normal(mlp.N_PARAMS)
    th2, m2, v2 = mlp.adamw_step(theta, g, np.zeros_like(g), np.zeros_like(g), 1, lr, wd)
    pad = ~mlp.active_mask()
    assert pad.sum() == 256 * 12
    assert np.all(th2[pad] == theta[pad]) and np.all(m2[pad] == 0) and np.all(v2[pad] == 0)


def test_adamw_first_step_closed_form():
    """At t = 1 from zero moments, m^ = g and v^ = g^2, so the step is
    lr g/(|g| + eps) plus the decay lr wd theta on weights only."""
    rng = np.random.default_rng(9)
    theta = mlp.init(5)
    g = rng.standard_normal(mlp.N_PARAMS) * 10.0 ** rng.uniform(-6, 0, mlp.N_PARAMS)
    lr, wd, eps = 1e-3, 0.1, 1e-8
    th, m, v = mlp.adamw_step(theta, g, np.zeros_like(g), np.zeros_like(g), 1, lr, wd, eps=eps)
    act = mlp.active_mask()
    expect = theta - lr * wd * mlp.decay_mask() * theta - lr * g / (np.abs(g) + eps)
    np.testing.assert_allclose(th[act], expect[act], rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(m[act], 0.1 * g[act], rtol=1e-12)
    np.testing.assert_allclose(v[act], 0.001 * g[act] ** 2, rtol=1e-12)
    # biases: no decay
    b1 = slice(256 * 16, 256 * 16 + 256)
    np.testing.assert_allclose(th[b1], theta[b1] - lr * g[b1] / (np.abs(g[b1]) + eps), rtol=1e-12)


def test_composition_bound_covers_fp32_and_catches_planted_mistakes():
    """The GPU gradient test's element-wise allowance (fp32 arithmetic bound
    without storage flips plus 2^-10 of each block's largest element) holds
    for an independent fp32 evaluation of the same storage scheme (PyTorch
    on the CPU, other summation order) and fails when a mistake is planted in
    that evaluation: one sign, two swapped rows, a transposed weight."""
    import os
    import sys
    import scipy.stats
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import mlp_error_bound as EB
    rng = np.random.default_rng(1)
    B = 300
    feats = rng.uniform(-1, 1, size=(B, 4)).astype(np.float32)
    lam = np.exp(2.0 + feats[:, 0] + 0.5 * feats[:, 2])
    t = scipy.stats.poisson.pmf(np.arange(128)[None, :], lam[:, None])
    t[:, -1] += 1.0 - t.sum(axis=1)
    t = t.astype(np.float32)
    theta = mlp.init(7).astype(np.float32).astype(np.float64)
    q, loss, g, Dq, Dg = EB.bounds(theta, feats.astype(np.float64), t.astype(np.float64), flips=False)

    def violations(gg):
        n_bad, at = 0, 0
        for name, shape in mlp.SHAPES:
            n = int(np.prod(shape))
            b = g[at:at + n]
            n_bad += int(np.sum(np.abs(gg[at:at + n] - b) > Dg[at:at + n] + 2.0**-10 * np.abs(b).max()))
            at += n
        return n_bad

    qe, ge = EB.fp32_emulation(theta, feats, t)
    assert np.all(np.abs(qe - q) <= Dq + 2.0**-10 * q.max(axis=1, keepdims=True))
    assert violations(ge) == 0
    for plant in ("sign", "swap", "transpose"):
        assert violations(EB.fp32_emulation(theta, feats, t, plant=plant)[1]) > 0, plant


def test_expected_w1_noise_matches_monte_carlo():
    """The check's sampling-noise estimate against brute force: the mean W1
    between a law and many n-draw empirical histograms of it (Poisson and
    bimodal laws on 0..127, n = 64 and 1024) within 5%."""
    import scipy.stats
    rng = np.random.default_rng(3)
    k = np.arange(128)
    laws = [scipy.stats.poisson.pmf(k, 20.0), 0.5 * scipy.stats.poisson.pmf(k, 3.0) + 0.5 * scipy.stats.poisson.pmf(k, 60.0)]
    for p in laws:
        p = p / p.sum()
        for n in (64, 1024):
            draws = rng.multinomial(n, p, size=4000) / n
            mc = mlp.wasserstein_hist(draws, p[None, :]).mean()
            est = float(mlp.expected_w1_noise(p[None, :], n)[0])
            assert abs(est - mc) <= 0.05 * mc, (n, est, mc)
