"""CPU oracle for the surrogate network (test infrastructure only).

A plain numpy float64 implementation of the telegraph surrogate: inputs are
4 standardised log-parameters (log kon, log koff, log km, log gamma) padded
with zeros to 16, three hidden layers of 256 GELU units, 128 output logits, a
softmax over mRNA counts 0..127 and the cross-entropy against an empirical
histogram p:  L = -(1/B) sum_b sum_k p_bk log softmax(z_b)_k.

GELU is the exact form x * Phi(x) with Phi the standard normal CDF.

The optimiser is AdamW (Loshchilov & Hutter, "Decoupled Weight Decay
Regularization", ICLR 2019, Algorithm 2 with the Adam bias corrections):
m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;  m^ = m/(1-b1^t);
v^ = v/(1-b2^t);  theta = theta - lr wd theta - lr m^/(sqrt(v^) + eps),
the decay term only on weight matrices (not biases), and the W1 padding
columns never touched.  The paper trains no network; this is the
surrogate's optimiser.

Parameter vector (float32 on the GPU, float64 here), in this order:
  W1 [256][16] (input columns 4..15 are padding and stay zero), b1 [256],
  W2 [256][256], b2 [256], W3 [256][256], b3 [256], W4 [128][256], b4 [128].

With ``bf16=True`` the values the GPU stores in bfloat16 are rounded to
bfloat16 at the same points (inputs, weights, hidden activations, and the
back-propagated pre-activation gradients that feed the GEMMs); all
arithmetic stays float64, so this is the exact result of the GPU's storage
scheme without its summation-order rounding.
"""
from __future__ import annotations

import numpy as np
import scipy.special

SHAPES = [("W1", (256, 16)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (256, 256)),
          ("b3", (256,)), ("W4", (128, 256)), ("b4", (128,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(theta):
    out, at = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[at:at + n], dtype=np.float64).reshape(shape)
        at += n
    return out


def flatten(params):
    return np.concatenate([np.asarray(params[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init(seed=0):
    """He-normal weights (std sqrt(2/fan_in), fan_in 4 for the first layer), zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SHAPES:
        if name.startswith("W"):
            fan_in = 4 if name == "W1" else shape[1]
            w = rng.standard_normal(shape) * np.sqrt(2.0 / fan_in)
            if name == "W1":
                w[:, 4:] = 0.0
            p[name] = w
        else:
            p[name] = np.zeros(shape)
    return flatten(p)


def bf16_round(x):
    """Round float64 values to bfloat16 (via float32, each step to nearest-even)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(torch.float32).to(torch.bfloat16)
    return t.to(torch.float64).numpy()


def gelu(z):
    return z * 0.5 * (1.0 + scipy.special.erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + scipy.special.erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def softmax(z):
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def forward(theta, features, bf16=False):
    """Returns (probabilities [B][128], cache)."""
    P = unflatten(theta)
    r = bf16_round if bf16 else (lambda a: a)
    B = features.shape[0]
    x = np.zeros((B, 16))
    x[:, :4] = features
    x = r(x)
    acts, zs = [x], []
    h = x
    for l in (1, 2, 3):
        z = h @ r(P[f"W{l}"]).T + P[f"b{l}"]
        zs.append(z)
        h = r(gelu(z))
        acts.append(h)
    logits = h @ r(P["W4"]).T + P["b4"]
    return softmax(logits), {"acts": acts, "zs": zs, "logits": logits, "P": P}


def loss_and_grad(theta, features, targets, bf16=False, trace=None):
    """Cross-entropy loss and its gradient with respect to theta.

    With a dict as ``trace``, the backward pass's intermediates are stored in
    it: q (probabilities), cache (the forward cache), and per layer l the
    pre-activation gradient dz{l} (l = 4 for the logits), its stored copy
    dzr{l} and the back-propagated dh{l} (l = 1..3)."""
    r = bf16_round if bf16 else (lambda a: a)
    q, c = forward(theta, features, bf16)
    P = c["P"]
    B = features.shape[0]
    loss = float(-(targets * np.log(np.maximum(q, 1e-300))).sum() / B)
    tr = trace if trace is not None else {}
    tr["q"], tr["cache"] = q, c
    g = {}
    dz = (q - targets) / B                      # d loss / d logits
    g["b4"] = dz.sum(axis=0)
    dz_r = r(dz)
    tr["dz4"], tr["dzr4"] = dz, dz_r
    g["W4"] = dz_r.T @ c["acts"][3]
    dh = dz_r @ r(P["W4"])
    for l in (3, 2, 1):
        tr[f"dh{l}"] = dh
        dz = dh * gelu_grad(c["zs"][l - 1])
        g[f"b{l}"] = dz.sum(axis=0)
        dz_r = r(dz)
        tr[f"dz{l}"], tr[f"dzr{l}"] = dz, dz_r
        g[f"W{l}"] = dz_r.T @ c["acts"][l - 1]
        if l > 1:
            dh = dz_r @ r(P[f"W{l}"])
    g["W1"][:, 4:] = 0.0
    return loss, flatten(g)


def wasserstein_hist(p, q):
    """W1 between two histograms on the integers 0..K-1 (rows)."""
    return np.abs(np.cumsum(p, axis=-1) - np.cumsum(q, axis=-1)).sum(axis=-1)


def decay_mask():
    """1 where AdamW applies weight decay (weight matrices), 0 for biases."""
    return np.concatenate([np.full(int(np.prod(shape)), 1.0 if name.startswith("W") else 0.0)
                           for name, shape in SHAPES])


def active_mask():
    """False for the W1 padding columns 4..15, which AdamW leaves alone."""
    a = np.ones(N_PARAMS, dtype=bool)
    a[:256 * 16] = np.tile(np.arange(16) < 4, 256)
    return a


def adamw_step(theta, grad, m, v, t, lr, wd, beta1=0.9, beta2=0.999, eps=1e-8):
    """One AdamW step (t = index of this step, starting at 1), float64.
    Returns (theta, m, v) after the step."""
    theta, grad, m, v = (np.asarray(a, dtype=np.float64) for a in (theta, grad, m, v))
    act = active_mask()
    m_new = np.where(act, beta1 * m + (1.0 - beta1) * grad, m)
    v_new = np.where(act, beta2 * v + (1.0 - beta2) * grad * grad, v)
    m_hat = m_new / (1.0 - beta1 ** t)
    v_hat = v_new / (1.0 - beta2 ** t)
    step = lr * m_hat / (np.sqrt(v_hat) + eps)
    th = theta - lr * wd * decay_mask() * theta - step
    return np.where(act, th, theta), m_new, v_new


def expected_w1_noise(p, n):
    """Expected W1 between the law p (rows, on the integers 0..K-1) and the
    empirical histogram of n draws from it: sum_k E|F_n(k) - F(k)|, each term
    by the normal approximation sqrt(2 F(k)(1 - F(k)) / (pi n)) of the mean
    absolute deviation of a binomial(n, F(k)) proportion."""
    p = np.asarray(p, dtype=np.float64)
    F = np.cumsum(p, axis=-1)
    rest = np.maximum(F[..., -1:] - F, 0.0)          # 1 - F as the remaining mass
    return np.sqrt(2.0 * np.maximum(F[..., :-1], 0.0) * rest[..., :-1] / (np.pi * n)).sum(axis=-1)
