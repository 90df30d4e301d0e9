"""Tensor-core (tcgen05) GEMM and surrogate-network kernels against plain
fp32 PyTorch references on the same bf16 inputs."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ssa():
    from paper_2605_00479_gb300 import build, ssa as mod
    build.build()
    mod.lib()
    return mod


@pytest.mark.parametrize("M,N,K", [(128, 16, 16), (300, 256, 256), (257, 128, 512), (1024, 256, 16), (64, 64, 32),
                                   (384, 16, 768), (200, 192, 64), (130, 144, 48), (256, 256, 2048),
                                   (300, 240, 512), (129, 208, 768)])
def test_gemm_matches_fp32_reference(ssa, M, N, K):
    """D = A B^T with bf16 operands and fp32 accumulation; the reference sums
    the same bf16 products in fp32 (differences come only from summation
    order: |err| <= K * 2^-23 * sum|a||b|).  K > 256 runs the two-stage
    pipeline (copies of one chunk under the MMAs of the previous), except
    where two stages of a wide column tile exceed shared memory (N = 240,
    208: one stage)."""
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = torch.full((M, N), float("nan"), device="cuda")
    rc = ssa.lib().ssa_mlp_gemm_bf16(M, N, K, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                     ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    ref = A.double() @ B.double().T
    bound = K * 2.0 ** -23 * (A.double().abs() @ B.double().abs().T) + 1e-30
    err = (D.double() - ref).abs()
    assert torch.all(err <= bound), float((err / bound).max())


def _features_targets(B, seed):
    rng = np.random.default_rng(seed)
    feats = rng.uniform(-1, 1, size=(B, 4)).astype(np.float32)
    lam = np.exp(2.0 + feats[:, 0] + 0.5 * feats[:, 2])          # a smooth family of laws
    k = np.arange(128)
    import scipy.stats
    t = scipy.stats.poisson.pmf(k[None, :], lam[:, None])
    t[:, -1] += 1.0 - t.sum(axis=1)
    return feats, t.astype(np.float32)


def _bf16_dev(a):
    """float64 array of bf16 values -> CUDA bf16 tensor (exact)."""
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda().to(torch.bfloat16)


def _bits(t):
    return t.cpu().view(torch.int16).numpy().view(np.uint16)


def _bf16_vals(t):
    return t.float().cpu().numpy().astype(np.float64)


def _assert_in_interval(name, got, iv, max_mismatch=1e-3):
    """Every stored bf16 value within its interval [lo, hi] (exactly the
    oracle's value where lo == hi).  The interval comes from worst-case fp32
    summation (gamma(K)), which at K = 256 admits the neighbour for a large
    share of elements; so the values that actually differ from the oracle's
    own rounding must also be rare (measured ~1e-4 for an fp32 emulation)."""
    lo, hi, mid = iv
    ok = (got >= lo) & (got <= hi)
    assert ok.all(), (name, int((~ok).sum()), np.argwhere(~ok)[:5])
    mismatch = float(np.mean(got != mid))
    assert mismatch <= max_mismatch, (name, mismatch)
    return mismatch


def _oracle_network(seed=7, B=300):
    """Oracle forward/backward at a He-initialised network: the stage inputs."""
    from oracle import mlp
    theta = mlp.init(seed).astype(np.float32).astype(np.float64)
    feats, t = _features_targets(B, 1)
    tr = {}
    mlp.loss_and_grad(theta, feats.astype(np.float64), t.astype(np.float64), bf16=True, trace=tr)
    return theta, feats, t, tr


@pytest.mark.parametrize("layer", [1, 2, 3])
def test_stage_hidden_forward_elementwise(ssa, layer):
    """Hidden-layer GEMM with the fused bias + GELU epilogue on the oracle's
    own bf16 activations and weights: z within the fp32 summation bound
    gamma(K) sum|a||w| + 2u|z| of the float64 value, and the stored bf16 GELU
    exactly the oracle's except where that bound straddles a rounding
    boundary (then one of the two neighbours)."""
    import mlp_error_bound as EB
    from oracle import mlp
    theta, feats, t, tr = _oracle_network()
    P = tr["cache"]["P"]
    A = tr["cache"]["acts"][layer - 1]
    W = mlp.bf16_round(P[f"W{layer}"])
    bias = P[f"b{layer}"].astype(np.float32).astype(np.float64)
    M, K = A.shape
    N = W.shape[0]
    z = torch.full((M, N), float("nan"), device="cuda")
    h = torch.zeros((M, N), dtype=torch.bfloat16, device="cuda")
    b_d = torch.from_numpy(bias.astype(np.float32)).cuda()
    A_d, W_d = _bf16_dev(A), _bf16_dev(W)      # kept alive until the synchronous call returns
    rc = ssa.lib().ssa_mlp_gemm_epi(1, M, N, K, ssa._dev_ptr(A_d), ssa._dev_ptr(W_d),
                                    ssa._dev_ptr(b_d), None, ssa._dev_ptr(z), ssa._dev_ptr(h), None, None)
    assert rc == 0
    z_o, Dz, iv = EB.stage_hidden_forward(A, W, bias)
    zg = z.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(zg - z_o) <= Dz), float((np.abs(zg - z_o) / Dz).max())
    _assert_in_interval("h", _bf16_vals(h), iv)


def test_stage_logits_elementwise(ssa):
    import mlp_error_bound as EB
    from oracle import mlp
    theta, feats, t, tr = _oracle_network()
    P = tr["cache"]["P"]
    A = tr["cache"]["acts"][3]
    W = mlp.bf16_round(P["W4"])
    bias = P["b4"].astype(np.float32).astype(np.float64)
    M, K = A.shape
    L = torch.full((M, 128), float("nan"), device="cuda")
    b_d = torch.from_numpy(bias.astype(np.float32)).cuda()
    A_d, W_d = _bf16_dev(A), _bf16_dev(W)
    rc = ssa.lib().ssa_mlp_gemm_epi(2, M, 128, K, ssa._dev_ptr(A_d), ssa._dev_ptr(W_d),
                                    ssa._dev_ptr(b_d), None, ssa._dev_ptr(L), None, None, None)
    assert rc == 0
    L_o, DL = EB.stage_logits(A, W, bias)
    assert np.all(np.abs(L.cpu().numpy() - L_o) <= DL)


def test_stage_softmax_cross_entropy_elementwise(ssa):
    """Softmax, (q - p)/B stored bf16, output-bias gradient and loss on the
    oracle's logits (rounded to fp32, the kernel's input type)."""
    import mlp_error_bound as EB
    theta, feats, t, tr = _oracle_network()
    L = tr["cache"]["logits"].astype(np.float32).astype(np.float64)
    B = L.shape[0]
    p = t.astype(np.float64)
    L_d = torch.from_numpy(L.astype(np.float32)).cuda()
    p_d = torch.from_numpy(t).cuda()
    dz = torch.zeros((B, 128), dtype=torch.bfloat16, device="cuda")
    bg = torch.zeros(128, device="cuda")
    loss = torch.zeros(1, device="cuda")
    probs = torch.full((B, 128), float("nan"), device="cuda")
    lib = ssa.lib()
    assert lib.ssa_mlp_softmax_xent(B, ssa._dev_ptr(L_d), None, ssa._dev_ptr(probs), None, None, None, None) == 0
    assert lib.ssa_mlp_softmax_xent(B, ssa._dev_ptr(L_d), ssa._dev_ptr(p_d), None, ssa._dev_ptr(dz),
                                    ssa._dev_ptr(bg), ssa._dev_ptr(loss), None) == 0
    q, Dq, iv, bg_o, Dbg, loss_o, Dloss = EB.stage_softmax_xent(L, p)
    assert np.all(np.abs(probs.cpu().numpy() - q) <= Dq)
    _assert_in_interval("dz", _bf16_vals(dz), iv)
    assert np.all(np.abs(bg.cpu().numpy() - bg_o) <= Dbg)
    assert abs(float(loss) - loss_o) <= Dloss


@pytest.mark.parametrize("layer", [3, 2])
def test_stage_hidden_backward_elementwise(ssa, layer):
    """Back-propagation GEMM with the fused GELU-derivative epilogue and the
    bias-gradient reduction: dz_l = (dz_{l+1} W_{l+1}) * gelu'(z_l) on the
    oracle's stored gradients, weights and pre-activations."""
    import mlp_error_bound as EB
    from oracle import mlp
    theta, feats, t, tr = _oracle_network()
    P = tr["cache"]["P"]
    A = tr[f"dzr{layer + 1}"]                                   # bf16 [B][K]
    Bm = np.ascontiguousarray(mlp.bf16_round(P[f"W{layer + 1}"]).T)   # [N][K]: W^T
    zin = tr["cache"]["zs"][layer - 1].astype(np.float32).astype(np.float64)
    M, K = A.shape
    N = Bm.shape[0]
    h = torch.zeros((M, N), dtype=torch.bfloat16, device="cuda")
    bg = torch.zeros(N, device="cuda")
    z_d = torch.from_numpy(zin.astype(np.float32)).cuda()
    A_d, B_d = _bf16_dev(A), _bf16_dev(Bm)
    rc = ssa.lib().ssa_mlp_gemm_epi(3, M, N, K, ssa._dev_ptr(A_d), ssa._dev_ptr(B_d), None,
                                    ssa._dev_ptr(z_d), None, ssa._dev_ptr(h), ssa._dev_ptr(bg), None)
    assert rc == 0
    iv, bg_o, Dbg = EB.stage_hidden_backward(A, Bm, zin)
    _assert_in_interval("dz", _bf16_vals(h), iv)
    assert np.all(np.abs(bg.cpu().numpy() - bg_o) <= Dbg)


def test_stage_weight_gradient_elementwise(ssa):
    """dW = dz^T h with the batch as the reduction (K = 512, two stages of the
    pipeline) on the oracle's stored values."""
    import mlp_error_bound as EB
    theta, feats, t, tr = _oracle_network(B=512)
    dzr = tr["dzr2"]                              # [512][256]
    h = tr["cache"]["acts"][1]                    # [512][256]
    A = np.ascontiguousarray(dzr.T)               # [256][512]
    Bm = np.ascontiguousarray(h.T)                # [256][512]
    D = torch.full((256, 256), float("nan"), device="cuda")
    A_d, B_d = _bf16_dev(A), _bf16_dev(Bm)
    assert ssa.lib().ssa_mlp_gemm_bf16(256, 256, 512, ssa._dev_ptr(A_d), ssa._dev_ptr(B_d), ssa._dev_ptr(D),
                                       None) == 0
    ref = A @ Bm.T
    bound = EB._gamma(512) * (np.abs(A) @ np.abs(Bm).T) + 1e-45
    assert np.all(np.abs(D.cpu().numpy() - ref) <= bound)


def test_surrogate_forward_and_gradients_match_oracle(ssa):
    """The whole training step's forward pass and gradient, element by
    element, against the float64 oracle with bf16 storage at the same points.
    Every fused stage is checked alone above, with bounds that follow from
    fp32 arithmetic; composed, a stored bf16 value can round the other way
    where the fp32 and float64 paths straddle a rounding boundary, and such
    one-ulp (2^-8 relative) flips cascade through the later layers.  The bound
    per element is therefore the fp32 arithmetic bound without flips plus
    2^-10 of the largest element of its parameter block (flip cascades measured
    at up to 1e-4 of it): a wrong sign, a transposed operand or a misplaced
    row moves an element by about its own size and fails."""
    import mlp_error_bound as EB
    from oracle import mlp
    net = ssa.Surrogate(max_batch=1024, seed=7)
    theta = net.get_params().astype(np.float64)
    assert theta.size == mlp.N_PARAMS and np.all(mlp.unflatten(theta)["W1"][:, 4:] == 0)
    B = 300
    feats, t = _features_targets(B, 1)
    f_d, t_d = torch.from_numpy(feats).cuda(), torch.from_numpy(t).cuda()
    probs = net.predict(f_d).cpu().numpy()
    loss, g = net.gradients(f_d, t_d)
    q, lo, go, Dq, Dg = EB.bounds(theta, feats.astype(np.float64), t.astype(np.float64), flips=False)
    # a flip in a hidden activation moves that row's logits, so each
    # probability gets 2^-6 of itself (fp32 emulations: up to 2.2e-3)
    dq = np.abs(probs - q) / (Dq + 2.0**-6 * q)
    assert np.all(dq <= 1.0), float(dq.max())
    assert abs(loss - lo) < 1e-3 * max(1.0, abs(lo))
    at = 0
    for name, shape in mlp.SHAPES:
        n = int(np.prod(shape))
        a, b, d = g[at:at + n].astype(np.float64), go[at:at + n], Dg[at:at + n]
        allow = d + 2.0**-10 * np.abs(b).max()
        bad = np.abs(a - b) > allow
        assert not bad.any(), (name, int(bad.sum()), float((np.abs(a - b) / allow).max()))
        at += n
    pad = mlp.unflatten(g.astype(np.float64))["W1"][:, 4:]
    assert np.all(pad == 0.0)
    net.status()


def test_adamw_update_matches_oracle_elementwise(ssa):
    """ssa_surrogate_train_step's AdamW update of theta, m and v against the
    oracle's AdamW (float64) applied to the same step's inputs: the state
    before the step, the gradient the step used and the step count, with the
    hyperparameters the kernel uses (beta1 = 0.9f, beta2 = 0.999f,
    eps = 1e-8f, binary32 lr and weight decay).  The kernel's fp32 update
    differs only by rounding, bounded operation by operation (u = 2^-24,
    first order: m, v, the bias corrections, sqrt, division, the decay),
    element by element; the W1 padding never moves."""
    from oracle import mlp
    f32 = lambda x: float(np.float32(x))   # noqa: E731
    b1, b2, eps = f32(0.9), f32(0.999), f32(1e-8)
    net = ssa.Surrogate(max_batch=256, seed=5)
    feats, t = _features_targets(256, 3)
    f_d, t_d = torch.from_numpy(feats).cuda(), torch.from_numpy(t).cuda()
    lr, wd = f32(2e-3), f32(0.01)
    for _ in range(3):                       # nonzero moments first
        net.train_step(f_d, t_d, lr, wd)
    th0, m0, v0, _, steps0 = net.get_state()
    net.train_step(f_d, t_d, lr, wd)
    th1, m1, v1, g, steps1 = net.get_state()
    assert steps1 == steps0 + 1 == 4
    D = lambda a: a.astype(np.float64)   # noqa: E731
    th_o, m_o, v_o = mlp.adamw_step(D(th0), D(g), D(m0), D(v0), steps1, lr, wd, b1, b2, eps)
    u = 2.0**-24
    act = mlp.active_mask()
    m0d, v0d, gd, t0d = D(m0), D(v0), D(g), D(th0)
    # first-order rounding bounds of the fp32 update, operation by operation
    Dm = 3 * u * (b1 * np.abs(m0d) + (1 - b1) * np.abs(gd)) + 1e-45
    Dv = 4 * u * (b2 * v0d + (1 - b2) * gd * gd) + 1e-45
    bc1, bc2 = 1 - b1 ** steps1, 1 - b2 ** steps1
    mhat, vhat = m_o / bc1, v_o / bc2
    Dmhat = (Dm + 2 * u * np.abs(m_o)) / bc1
    Dvhat = (Dv + 2 * u * v_o) / bc2
    s_ = np.sqrt(vhat)
    Ds = np.minimum(Dvhat / (2 * np.maximum(s_, 1e-300)), np.sqrt(Dvhat)) + u * s_
    den = s_ + eps
    step = lr * mhat / den
    Dstep = lr * Dmhat / den + np.abs(step) * (Ds + u * den) / den + 3 * u * np.abs(step)
    decay = lr * wd * np.abs(t0d)
    Dt = 3 * u * decay + u * np.abs(t0d) + Dstep + u * np.abs(th_o) + 1e-45
    for name, got, exp, bnd in (("m", m1, m_o, Dm), ("v", v1, v_o, Dv), ("theta", th1, th_o, Dt)):
        err = np.abs(D(got) - exp)
        assert np.all(err[act] <= bnd[act]), (name, float((err[act] / bnd[act]).max()))
    # the bound is tight: a step with the wrong sign, no bias correction or
    # decay on biases would exceed it by orders of magnitude
    assert np.median(Dt[act] / np.maximum(np.abs(step[act]), 1e-30)) < 1e-4
    assert np.all(th1[~act] == 0) and np.all(m1[~act] == 0) and np.all(v1[~act] == 0)
    # the update is not trivial: every active parameter moved
    assert np.mean(th1[act] != th0[act]) > 0.99


def test_gemm_waits_that_run_out_report_timeouts(ssa):
    """Failure detection of the tensor-core GEMM: with the operand loads (1)
    or the MMAs (2) withheld, the bounded wait runs out, the kernel records
    its error word, drains and returns, and the call reports SSA_ETIMEDOUT;
    the context stays usable.  A short bound without withholding gives either
    SSA_ETIMEDOUT or a correct result, never a silent wrong one."""
    lib = ssa.lib()
    g = torch.Generator(device="cuda").manual_seed(3)
    A = torch.randn(256, 256, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(128, 256, device="cuda", generator=g).to(torch.bfloat16)
    ref = A.double() @ B.double().T
    bound = 256 * 2.0 ** -23 * (A.double().abs() @ B.double().abs().T) + 1e-30

    def gemm():
        D = torch.full((256, 128), float("nan"), device="cuda")
        rc = lib.ssa_mlp_gemm_bf16(256, 128, 256, ssa._dev_ptr(A), ssa._dev_ptr(B), ssa._dev_ptr(D), None)
        return rc, D

    try:
        for withhold, limit in ((1, 1000), (2, 1 << 16)):
            assert lib.ssa_mlp_set_wait_test(withhold, limit) == 0
            rc, _ = gemm()
            assert rc == ssa.SSA_ETIMEDOUT, (withhold, rc)
        assert lib.ssa_mlp_set_wait_test(0, 1) == 0
        for _ in range(3):
            rc, D = gemm()
            assert rc in (ssa.SSA_OK, ssa.SSA_ETIMEDOUT)
            if rc == ssa.SSA_OK:
                assert torch.all((D.double() - ref).abs() <= bound)
        # the surrogate's error word comes back through ssa_surrogate_status
        assert lib.ssa_mlp_set_wait_test(0, 0) == 0
        net = ssa.Surrogate(max_batch=256, seed=1)
        feats, _ = _features_targets(256, 4)
        f_d = torch.from_numpy(feats).cuda()
        assert lib.ssa_mlp_set_wait_test(1, 1000) == 0
        net.predict(f_d)
        with pytest.raises(ssa.SSAError) as exc:
            net.status()
        assert exc.value.code == ssa.SSA_ETIMEDOUT
    finally:
        lib.ssa_mlp_set_wait_test(0, 0)
    rc, D = gemm()
    assert rc == ssa.SSA_OK and torch.all((D.double() - ref).abs() <= bound)
    net2 = ssa.Surrogate(max_batch=256, seed=1)
    net2.predict(f_d)
    net2.status()
    assert lib.ssa_mlp_set_wait_test(3, 0) == ssa.SSA_EINVAL


def test_surrogate_training_reduces_loss(ssa):
    net = ssa.Surrogate(max_batch=512, seed=3)
    feats, t = _features_targets(4096, 2)
    f_d, t_d = torch.from_numpy(feats).cuda(), torch.from_numpy(t).cuda()
    loss = torch.zeros(1, device="cuda")
    first = None
    for step in range(400):
        i = (step * 512) % 4096
        net.train_step(f_d[i:i + 512], t_d[i:i + 512], lr=1e-3, loss=loss)
        if step == 0:
            torch.cuda.synchronize()
            first = float(loss)
    torch.cuda.synchronize()
    last = float(loss)
    net.status()
    entropy = float(-(t * np.log(np.maximum(t, 1e-30))).sum(axis=1).mean())
    assert last < first and (last - entropy) < 0.25 * (first - entropy), (first, last, entropy)


def test_histogram_and_w1_kernels(ssa):
    rng = np.random.default_rng(4)
    counts = rng.poisson(20, size=(37, 300)).astype(np.int32)
    counts[0, :5] = 500       # clamped into the last bin
    c_d = torch.from_numpy(counts).cuda().reshape(-1)
    h = ssa.histogram(c_d, 37, 300).cpu().numpy()
    ref = np.stack([np.bincount(np.minimum(r, 127), minlength=128) / 300.0 for r in counts])
    np.testing.assert_allclose(h, ref, rtol=0, atol=1e-7)
    q = np.roll(ref, 1, axis=1)
    w = ssa.hist_w1(torch.from_numpy(ref.astype(np.float32)).cuda(), torch.from_numpy(q.astype(np.float32)).cuda())
    from oracle import mlp
    np.testing.assert_allclose(w.cpu().numpy(), mlp.wasserstein_hist(ref, q), rtol=1e-4, atol=1e-5)


def test_w1_noise_kernel_matches_oracle(ssa):
    """ssa_hist_w1_noise against the oracle's expected_w1_noise (fp32 prefix
    sums and square roots vs float64: 1e-4 relative)."""
    from oracle import mlp
    rng = np.random.default_rng(8)
    p = rng.random((300, 128)) ** 4
    p[:5, 40:] = 0.0                              # laws with empty tails
    p /= p.sum(axis=1, keepdims=True)
    for n in (64, 1000):
        got = ssa.hist_w1_noise(torch.from_numpy(p.astype(np.float32)).cuda(), n).cpu().numpy()
        np.testing.assert_allclose(got, mlp.expected_w1_noise(p.astype(np.float32).astype(np.float64), n),
                                   rtol=1e-4, atol=1e-6)


def test_graph_driven_training_matches_step_by_step(ssa):
    """ssa_surrogate_train (one captured step replayed) against the same steps
    issued one by one through ssa_surrogate_train_step with the documented
    minibatches and learning rates.  Bias gradients are summed with fp32
    atomics, so the two runs agree up to that summation order: losses to 1e-5
    relative; parameters to 1e-5 except a small fraction (AdamW's normalised
    step turns a last-bit difference in a near-zero gradient into a difference
    of up to 2 lr per step)."""
    import math
    n, B, steps, lr_max, lr_min, wd = 3000, 256, 12, 2e-3, 5e-5, 1e-4
    rng = np.random.default_rng(3)
    feats = torch.from_numpy(rng.normal(size=(n, 4)).astype(np.float32)).cuda()
    t = rng.random((n, 128)).astype(np.float32)
    t /= t.sum(axis=1, keepdims=True)
    targs = torch.from_numpy(t).cuda()
    a = ssa.Surrogate(B, seed=7)
    b = ssa.Surrogate(B, seed=7)
    np.testing.assert_array_equal(a.get_params(), b.get_params())
    trace = torch.full((steps,), float("nan"), device="cuda")
    a.train(feats, targs, steps, B, lr_max, lr_min, wd, loss_every=1, loss_trace=trace)
    loss = torch.zeros(1, device="cuda")
    losses = []
    for k in range(steps):
        rows = torch.from_numpy((k * B + np.arange(B)) % n).cuda()
        lr = lr_min + 0.5 * (lr_max - lr_min) * (1 + math.cos(math.pi * k / (steps - 1)))
        b.train_step(feats[rows], targs[rows], lr, wd, loss=loss)
        losses.append(float(loss))
    np.testing.assert_allclose(trace.cpu().numpy(), np.array(losses, np.float32), rtol=1e-5)
    assert losses[-1] < losses[0]
    pa, pb = a.get_params(), b.get_params()
    d = np.abs(pa - pb)
    assert np.mean(d <= 1e-5 + 1e-5 * np.abs(pb)) > 0.99
    assert d.max() <= 2 * lr_max * steps


def test_graph_driven_training_trace_every_and_validation(ssa):
    n, B = 1000, 128
    feats = torch.zeros((n, 4), device="cuda")
    targs = torch.full((n, 128), 1.0 / 128, device="cuda")
    s = ssa.Surrogate(B, seed=1)
    trace = torch.full((4,), float("nan"), device="cuda")
    s.train(feats, targs, 10, B, 1e-3, 1e-3, 0.0, loss_every=3, loss_trace=trace)   # steps 0, 3, 6, 9
    assert torch.isfinite(trace).all()
    with pytest.raises(ssa.SSAError):
        s.train(feats, targs, 5, B + 1, 1e-3, 1e-3)      # batch above max_batch
    with pytest.raises(ssa.SSAError):
        s.train(feats, targs, 5, B, 1e-3, 1e-3, loss_every=0)
