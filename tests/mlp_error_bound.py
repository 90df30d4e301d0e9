"""Element-wise error bounds for the surrogate network's forward pass and
gradients computed in fp32 with bf16 storage (test helper, not a test file).

The oracle (oracle/mlp.py) evaluates the network in float64 and rounds to
bfloat16 exactly where the tensor-core implementation stores bfloat16
(inputs, weights, hidden activations, back-propagated pre-activation
gradients).  An fp32 implementation of the same storage scheme differs from
it only through

* the order and precision of its fp32 sums: a K-term dot product of exact
  products carries at most gamma(K) = K 2^-23 times sum |a||b| (two units in
  the last place per addition, which also allows truncating adders), and
  each further fp32 operation one unit u = 2^-24 of its result;
* its fp32 GELU, GELU derivative, exp and division (a few units each);
* and what those differences do at a bf16 storage point: the stored value
  can change only where the interval [y - d, y + d] around the oracle's
  pre-rounding value y contains a rounding boundary, and then by at most
  r(y + d) - r(y - d) (rounding is monotone).

Propagating these first-order absolute bounds layer by layer gives a bound
per output element.  Where no stored value flips, the bound is a few ulps
of the fp32 sums; a wrong sign, a transposed operand or a swapped row moves
an element by about its own size and fails it.
"""
import numpy as np
import scipy.special

from oracle import mlp

U = 2.0 ** -24


def _gamma(K):
    return K * 2.0 ** -23


def _flip(y, d):
    """Largest change of the bf16-stored copy of y under a perturbation <= d."""
    return np.abs(mlp.bf16_round(y + d) - mlp.bf16_round(y - d))


def _phi(z):
    return np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def _Phi(z):
    return 0.5 * (1.0 + scipy.special.erf(z / np.sqrt(2.0)))


def bounds(theta, features, targets, flips=True):
    """Returns (q, loss, grad, bound_q, bound_grad) for a minibatch: the
    oracle's probabilities, loss and gradient (float64, bf16 storage) and the
    element-wise bounds on an fp32 implementation's deviation from them.
    flips=False drops every bf16 storage flip (the part of the bound that
    compounds through the layers) and keeps the fp32 arithmetic part."""
    r = mlp.bf16_round
    _fl = _flip if flips else (lambda y, d: np.zeros_like(y))
    tr = {}
    loss, grad = mlp.loss_and_grad(theta, features, targets, bf16=True, trace=tr)
    c = tr["cache"]
    P = c["P"]
    acts, zs = c["acts"], c["zs"]
    B = features.shape[0]
    Wr = {l: np.abs(r(P[f"W{l}"])) for l in (1, 2, 3, 4)}
    K = {1: 16, 2: 256, 3: 256, 4: 256}
    Bpad = (B + 255) // 256 * 256

    # forward: bounds on z, the stored activations h and the logits
    Dh = [np.zeros_like(acts[0])]              # the inputs are rounded identically on both sides
    Dz = []
    for l in (1, 2, 3):
        h, z = acts[l - 1], zs[l - 1]
        dz = _gamma(K[l]) * (np.abs(h) @ Wr[l].T) + Dh[-1] @ Wr[l].T + 2 * U * np.abs(z)
        Dz.append(dz)
        g = mlp.gelu(z)
        dg = 1.13 * dz + 8 * U * np.abs(z) + 1e-45
        Dh.append(_fl(g, dg))
    L = c["logits"]
    DL = _gamma(K[4]) * (np.abs(acts[3]) @ Wr[4].T) + Dh[3] @ Wr[4].T + 2 * U * np.abs(L)

    # softmax: relative error of each probability
    q = tr["q"]
    rel = DL + DL.max(axis=1, keepdims=True) + U * np.abs(L - L.max(axis=1, keepdims=True)) + 24 * U
    Dq = q * np.expm1(rel) * 1.01
    p = np.asarray(targets, dtype=np.float64)

    bound = {}
    dz4 = tr["dz4"]
    Ddz = (Dq * (1 + U) + 2 * U * np.abs(q - p)) / B + U * np.abs(dz4)
    bound["b4"] = Ddz.sum(axis=0) + _gamma(B) * np.abs(dz4).sum(axis=0)
    dzr = tr["dzr4"]
    Ddzr = _fl(dz4, Ddz)
    h = acts[3]
    bound["W4"] = (_gamma(Bpad) * (np.abs(dzr).T @ np.abs(h)) + Ddzr.T @ np.abs(h) + np.abs(dzr).T @ Dh[3]
                   + Ddzr.T @ Dh[3])
    Ddh = _gamma(128) * (np.abs(dzr) @ Wr[4]) + Ddzr @ Wr[4]
    for l in (3, 2, 1):
        z = zs[l - 1]
        dh = tr[f"dh{l}"]
        gp = mlp.gelu_grad(z)
        Dgp = 0.8 * Dz[l - 1] + U * (4 * _Phi(z) + (6 + 0.5 * z * z) * np.abs(z) * _phi(z) + np.abs(gp)) + 1e-45
        dz = tr[f"dz{l}"]
        Ddz = Ddh * np.abs(gp) + np.abs(dh) * Dgp + Ddh * Dgp + U * np.abs(dz)
        bound[f"b{l}"] = Ddz.sum(axis=0) + _gamma(B) * np.abs(dz).sum(axis=0)
        dzr = tr[f"dzr{l}"]
        Ddzr = _fl(dz, Ddz)
        h = acts[l - 1]
        bound[f"W{l}"] = (_gamma(Bpad) * (np.abs(dzr).T @ np.abs(h)) + Ddzr.T @ np.abs(h)
                          + np.abs(dzr).T @ Dh[l - 1] + Ddzr.T @ Dh[l - 1])
        if l > 1:
            Ddh = _gamma(256) * (np.abs(dzr) @ Wr[l]) + Ddzr @ Wr[l]
    bound["W1"][:, 4:] = 0.0
    return q, loss, grad, Dq, mlp.flatten(bound)


def fp32_emulation(theta, features, targets, plant=None):
    """The storage scheme evaluated in plain fp32 PyTorch on the CPU (another
    summation order, torch's own exp and erf): a second implementation the
    bound must cover.  ``plant`` injects a mistake to show the bound catches
    it: 'sign' (one dW4 element negated), 'swap' (two rows of dW2 swapped),
    'transpose' (W3^T in place of W3 in the backward pass)."""
    import torch
    f32 = torch.float32

    def r(a):
        return a.to(torch.bfloat16).to(f32)

    P = {k: torch.tensor(v, dtype=f32) for k, v in mlp.unflatten(np.asarray(theta, np.float32)).items()}
    B = features.shape[0]
    x = torch.zeros((B, 16), dtype=f32)
    x[:, :4] = torch.tensor(np.asarray(features, np.float32))
    x = r(x)
    acts, zs = [x], []
    h = x
    for l in (1, 2, 3):
        z = h @ r(P[f"W{l}"]).T + P[f"b{l}"]
        zs.append(z)
        h = r(0.5 * z * (1.0 + torch.erf(z * 0.70710678118654752)))
        acts.append(h)
    L = h @ r(P["W4"]).T + P["b4"]
    e = torch.exp(L - L.max(dim=1, keepdim=True).values)
    q = e / e.sum(dim=1, keepdim=True)
    t = torch.tensor(np.asarray(targets, np.float32))
    g = {}
    dz = (q - t) / B
    g["b4"] = dz.sum(dim=0)
    dzr = r(dz)
    g["W4"] = dzr.T @ acts[3]
    dh = dzr @ r(P["W4"])
    for l in (3, 2, 1):
        z = zs[l - 1]
        gp = 0.5 * (1.0 + torch.erf(z * 0.70710678118654752)) + z * 0.39894228040143268 * torch.exp(-0.5 * z * z)
        dz = dh * gp
        g[f"b{l}"] = dz.sum(dim=0)
        dzr = r(dz)
        g[f"W{l}"] = dzr.T @ acts[l - 1]
        if l > 1:
            Wl = r(P[f"W{l}"])
            if plant == "transpose" and l == 3:
                Wl = Wl.T.contiguous()
            dh = dzr @ Wl
    g["W1"][:, 4:] = 0.0
    if plant == "sign":   # the largest element of dW4
        i = int(torch.argmax(g["W4"].abs()))
        g["W4"].view(-1)[i] = -g["W4"].view(-1)[i]
    if plant == "swap":   # two rows of dW2
        g["W2"][[10, 11]] = g["W2"][[11, 10]]
    return q.numpy().astype(np.float64), mlp.flatten({k: v.numpy() for k, v in g.items()})


# ---------------------------------------------------------------- stage bounds
# Each fused kernel of the training step on given inputs (exact bf16 / fp32
# values): the float64 result and the element-wise bound of an fp32
# implementation.  A bf16 output must lie in [lo, hi] = [r(y - d), r(y + d)];
# where lo == hi (almost everywhere) that is one exact value.

def _interval(y, d):
    """(r(y - d), r(y + d), r(y)): the candidates' range and the oracle's own
    stored value."""
    r = mlp.bf16_round
    return r(y - d), r(y + d), r(y)


def stage_hidden_forward(A, W, bias):
    """z = A W^T + bias, h = bf16(gelu(z)): returns z, bound_z and the
    interval (lo, hi, oracle value) of h."""
    K = A.shape[1]
    z = A @ W.T + bias
    Dz = _gamma(K) * (np.abs(A) @ np.abs(W).T) + 2 * U * np.abs(z)
    return z, Dz, _interval(mlp.gelu(z), 1.13 * Dz + 8 * U * np.abs(z) + 1e-45)


def stage_logits(A, W, bias):
    K = A.shape[1]
    L = A @ W.T + bias
    return L, _gamma(K) * (np.abs(A) @ np.abs(W).T) + 2 * U * np.abs(L)


def stage_hidden_backward(A, B, zin):
    """d = (A B^T) gelu'(zin), h = bf16(d), bias_grad = column sums of d:
    returns the interval (lo, hi, oracle value) of h, bias_grad and its
    bound."""
    K = A.shape[1]
    acc = A @ B.T
    Dacc = _gamma(K) * (np.abs(A) @ np.abs(B).T)
    gp = mlp.gelu_grad(zin)
    Dgp = U * (4 * _Phi(zin) + (6 + 0.5 * zin * zin) * np.abs(zin) * _phi(zin) + np.abs(gp)) + 1e-45
    d = acc * gp
    Dd = Dacc * np.abs(gp) + np.abs(acc) * Dgp + Dacc * Dgp + U * np.abs(d)
    M = A.shape[0]
    return _interval(d, Dd), d.sum(axis=0), Dd.sum(axis=0) + _gamma(M) * np.abs(d).sum(axis=0)


def stage_softmax_xent(L, p):
    """q = softmax(L), dz = (q - p)/B stored bf16, bias_grad = sum of dz over
    rows, loss = mean cross-entropy: returns q, bound_q, the interval
    (lo, hi, oracle value) of dz, bias_grad, bound_bias_grad, loss,
    bound_loss."""
    B = L.shape[0]
    mx = L.max(axis=1, keepdims=True)
    e = np.exp(L - mx)
    q = e / e.sum(axis=1, keepdims=True)
    Dq = q * np.expm1(U * np.abs(L - mx) + 24 * U) * 1.01
    dz = (q - p) / B
    Ddz = (Dq * (1 + U) + 2 * U * np.abs(q - p)) / B + U * np.abs(dz)
    iv = _interval(dz, Ddz)
    lse = np.log(e.sum(axis=1, keepdims=True))
    terms = p * (L - mx - lse)
    loss = float(-terms.sum() / B)
    Dterm = p * (U * np.abs(L - mx) + (20 * U) * np.maximum(1.0, np.abs(lse))) + 4 * U * np.abs(terms)
    Dloss = float((Dterm.sum() + _gamma(128) * np.abs(terms).sum()) / B * (1 + _gamma(B)) + U * abs(loss))
    return (q, Dq, iv, dz.sum(axis=0), Ddz.sum(axis=0) + _gamma(B) * np.abs(dz).sum(axis=0), loss, Dloss)
