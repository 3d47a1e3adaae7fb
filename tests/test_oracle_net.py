"""Pins of the network oracle: a pure-Python loop convolution on tiny blocks,
central finite differences of the loss for every parameter group and the input,
and the Adam update against its scalar recurrence."""
import numpy as np
import pytest

from oracle import net


def _loop_conv(x, W, b):
    B, Cin, n = x.shape[0], x.shape[1], x.shape[-1]
    y = np.zeros((B, W.shape[0], n, n, n))
    for bb in range(B):
        for o in range(W.shape[0]):
            for k in range(n):
                for j in range(n):
                    for i in range(n):
                        s = b[o]
                        for c in range(Cin):
                            for t, (dk, dj, di) in enumerate(net.TAPS):
                                kk, jj, ii = k + dk, j + dj, i + di
                                if 0 <= kk < n and 0 <= jj < n and 0 <= ii < n:
                                    s += W[o, c, t] * x[bb, c, kk, jj, ii]
                        y[bb, o, k, j, i] = s
    return y


def test_conv_matches_loop_definition():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 4, 4, 4))
    W = rng.normal(size=(2, 3, 27))
    b = rng.normal(size=2)
    assert np.allclose(net.conv(x, W, b), _loop_conv(x, W, b), rtol=1e-13, atol=1e-13)


def test_conv_center_tap_is_pointwise_and_shift_is_exact():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 2, 5, 5, 5))
    W = np.zeros((1, 2, 27))
    W[0, 0, 13] = 2.0  # tap (0,0,0)
    W[0, 1, 14] = 1.0  # tap (0,0,+1): reads x[..., i+1]
    y = net.conv(x, W, np.zeros(1))[0, 0]
    expect = 2.0 * x[0, 0].copy()
    expect[:, :, :4] += x[0, 1][:, :, 1:]
    assert np.array_equal(y, expect)


def test_gelu_values_and_derivative():
    v = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    # Phi(0) = 1/2, gelu(0) = 0; gelu(x) - gelu(-x) = x (since Phi(x) + Phi(-x) = 1)
    assert net.gelu(np.array([0.0]))[0] == 0.0
    assert np.allclose(net.gelu(v) - net.gelu(-v), v, rtol=0, atol=1e-15)
    h = 1e-6
    fd = (net.gelu(v + h) - net.gelu(v - h)) / (2 * h)
    assert np.allclose(net.gelu_grad(v), fd, rtol=1e-8, atol=1e-9)


@pytest.mark.parametrize("n", [3, 4])
def test_gradients_by_central_differences(n):
    rng = np.random.default_rng(n)
    B = 2
    theta = rng.normal(scale=0.3, size=net.NPARAM)
    x = rng.normal(size=(B, net.CIN, n, n, n))
    t = rng.normal(size=(B, n, n, n))
    L, g, dx = net.loss_and_grad(theta, x, t)
    assert abs(L - net.loss(theta, x, t)) <= 1e-12 * L
    h = 1e-6
    # every parameter group, a few entries each
    o = 0
    for name, shp in net.SHAPES:
        size = int(np.prod(shp))
        for idx in rng.choice(size, size=min(size, 6), replace=False):
            e = np.zeros(net.NPARAM)
            e[o + idx] = h
            fd = (net.loss(theta + e, x, t) - net.loss(theta - e, x, t)) / (2 * h)
            assert abs(fd - g[o + idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, g[o + idx])
        o += size
    for _ in range(5):
        pos = tuple(rng.integers(0, s) for s in x.shape)
        e = np.zeros_like(x)
        e[pos] = h
        fd = (net.loss(theta, x + e, t) - net.loss(theta, x - e, t)) / (2 * h)
        assert abs(fd - dx[pos]) <= 1e-6 * max(1.0, abs(fd))


def test_adam_matches_scalar_recurrence():
    theta = np.array([1.0, -2.0])
    g = np.array([0.5, -0.25])
    m = np.zeros(2)
    v = np.zeros(2)
    th, m, v = net.adam(theta, g, m, v, 1, lr=0.1)
    # first step: mhat = g, vhat = g^2 -> step = lr * g / (|g| + eps) ~ lr * sign(g)
    assert np.allclose(th, theta - 0.1 * np.sign(g), rtol=0, atol=1e-7)


def test_element_inputs_normalisation():
    rng = np.random.default_rng(3)
    r = rng.normal(size=(4, 27)) * np.array([[1.0], [0.0], [5.0], [1e-3]])
    jr = r * 2.0
    x, sr, sj = net.element_inputs(r, jr)
    assert np.all(x[1] == 0.0) and sr[1] == 0.0
    for e in (0, 2, 3):
        assert abs(np.sqrt(np.mean(x[e, 0] ** 2)) - 1.0) < 1e-14
        assert abs(np.sqrt(np.mean(x[e, 1] ** 2)) - 1.0) < 1e-14


def test_energy_loss_gradient_by_central_differences():
    from oracle import ref
    from paper_2011_04981_gb300 import inputs

    n = 3
    rng = np.random.default_rng(9)
    mesh = inputs.box_mesh(2, 1, 1, n, perturb=0.2, seed=2)
    xi, rho, D = ref.gll(n)
    G = ref.geom(mesh.corners, n, xi, rho)
    A = np.stack([ref.element_matrix(D, G[e]) for e in range(2)])
    theta = rng.normal(scale=0.3, size=net.NPARAM)
    x = rng.normal(size=(2, net.CIN, n, n, n))
    t = rng.normal(size=(2, n, n, n))
    L, g, dx = net.energy_loss_and_grad(theta, x, t, A)
    assert abs(L - net.energy_loss(theta, x, t, A)) <= 1e-12 * L
    # constants are in the kernel of every element matrix: adding one to y changes nothing
    P = net.unpack(theta)
    P["b3"] = P["b3"] + 0.7
    assert abs(net.energy_loss(net.pack(P), x, t, A) - L) <= 1e-10 * L
    h = 1e-6
    o = 0
    for name, shp in net.SHAPES:
        size = int(np.prod(shp))
        for idx in rng.choice(size, size=min(size, 5), replace=False):
            e = np.zeros(net.NPARAM)
            e[o + idx] = h
            fd = (net.energy_loss(theta + e, x, t, A) - net.energy_loss(theta - e, x, t, A)) / (2 * h)
            assert abs(fd - g[o + idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx)
        o += size


def test_bf16_rounding_matches_torch_and_forward_rounds_activations():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    v = np.concatenate([rng.normal(scale=10.0 ** rng.uniform(-6, 6, 4000)), [0.0, -0.0, 1.0, -3.0, 65504.0],
                        # halfway cases between neighbouring BF16 values: ties go to even
                        [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8)]])
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(net.bf16_round(v), ref)
    assert net.bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert net.bf16_round(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    # with the identity as rounding, forward is unchanged; with BF16 it moves by a BF16-sized amount
    th = rng.normal(scale=0.25, size=net.NPARAM)
    x = rng.normal(size=(2, 2, 8, 8, 8))
    y = net.forward(th, x)
    assert np.array_equal(net.forward(th, x, act_round=lambda a: a), y)
    yb = net.forward(th, x, act_round=net.bf16_round)
    rel = np.linalg.norm(yb - y) / np.linalg.norm(y)
    assert 1e-4 < rel < 3e-2


# --- the componentwise rounding-error bounds, pinned to an FP32 evaluation -------
# A second evaluation of the network, written with explicit sequential FP32 sums
# (one tap and one channel at a time, as a GPU thread accumulates), stands in for
# any FP32 kernel: its difference from the FP64 oracle must stay inside the
# bound of every output and every gradient entry, and the bound must be tight
# enough (relative to the data) that a wrong entry cannot hide in it.

F32 = np.float32


def _conv32(x, W, b):
    x = x.astype(F32)
    W = W.astype(F32)
    y = np.broadcast_to(b.astype(F32)[None, :, None, None, None], (x.shape[0], W.shape[0]) + x.shape[2:]).copy()
    for t, (dk, dj, di) in enumerate(net.TAPS):
        xs = net.shift(x, dk, dj, di).astype(F32)
        for c in range(W.shape[1]):
            y = (y + (W[None, :, c, t, None, None, None] * xs[:, c:c + 1]).astype(F32)).astype(F32)
    return y


def _convT32(dy, W):
    dy = dy.astype(F32)
    W = W.astype(F32)
    dx = np.zeros((dy.shape[0], W.shape[1]) + dy.shape[2:], dtype=F32)
    for t, (dk, dj, di) in enumerate(net.TAPS):
        for o in range(W.shape[0]):
            s = net.shift(dy[:, o:o + 1], -dk, -dj, -di).astype(F32)
            dx = (dx + (W[None, o, :, t, None, None, None] * s).astype(F32)).astype(F32)
    return dx


def _wgrad32(dy, x):
    dW = np.zeros((dy.shape[1], x.shape[1], 27), dtype=F32)
    for t, (dk, dj, di) in enumerate(net.TAPS):
        xs = net.shift(x.astype(F32), dk, dj, di).astype(F32)
        for b in range(dy.shape[0]):
            dW[:, :, t] = (dW[:, :, t] + np.einsum("okji,ckji->oc", dy[b].astype(F32), xs[b]).astype(F32)).astype(F32)
    return dW


def _gelu32(v):
    return (F32(0.5) * v * (F32(1) + net.erf(v * F32(1 / np.sqrt(2))).astype(F32))).astype(F32)


def _forward32(theta, x, act_round=None):
    P = {k: v.astype(F32) for k, v in net.unpack(theta).items()}
    rnd = (lambda v: act_round(v).astype(F32)) if act_round else (lambda v: v.astype(F32))
    x0 = rnd(x)
    h1 = _conv32(x0, P["W1"], P["b1"])
    a1 = rnd(_gelu32(h1))
    h2 = _conv32(a1, P["W2"], P["b2"])
    a2 = rnd(_gelu32(h2))
    return _conv32(a2, P["W3"], P["b3"]), (x0, h1, a1, h2, a2)


def _backward32(theta, cache, dy):
    P = {k: v.astype(F32) for k, v in net.unpack(theta).items()}
    x0, h1, a1, h2, a2 = cache
    gp = lambda h: net.gelu_grad(h.astype(np.float64)).astype(F32)  # noqa: E731
    g = {"W3": _wgrad32(dy, a2), "b3": dy.sum(axis=(0, 2, 3, 4), dtype=F32)}
    dh2 = (_convT32(dy, P["W3"]) * gp(h2)).astype(F32)
    g["W2"], g["b2"] = _wgrad32(dh2, a1), dh2.sum(axis=(0, 2, 3, 4), dtype=F32)
    dh1 = (_convT32(dh2, P["W2"]) * gp(h1)).astype(F32)
    g["W1"], g["b1"] = _wgrad32(dh1, x0), dh1.sum(axis=(0, 2, 3, 4), dtype=F32)
    return net.pack({k: v.astype(np.float64) for k, v in g.items()})


def _grad32(theta, x, t):
    B = x.shape[0]
    y, cache = _forward32(theta, x)
    r = (y[:, 0] - t.astype(F32)).astype(F32)
    den = np.sum(t.astype(F32) ** 2, axis=(1, 2, 3), dtype=F32)
    dy = (F32(2.0 / B) * r / den[:, None, None, None])[:, None].astype(F32)
    return _backward32(theta, cache, dy)


def _energy_grad32(theta, x, t, A):
    B = x.shape[0]
    y, cache = _forward32(theta, x)
    A32 = A.astype(F32)
    d = (y[:, 0].reshape(B, -1) - t.reshape(B, -1).astype(F32)).astype(F32)
    Ad = np.einsum("bpq,bq->bp", A32, d).astype(F32)
    t32 = t.reshape(B, -1).astype(F32)
    den = np.sum(t32 * np.einsum("bpq,bq->bp", A32, t32).astype(F32), axis=1, dtype=F32)
    dy = (F32(2.0 / B) * Ad / den[:, None]).astype(F32).reshape(y.shape)
    return _backward32(theta, cache, dy)


def _theta(seed, scale=0.25):
    th = np.random.default_rng(seed).normal(scale=scale, size=net.NPARAM)
    return net.bf16_round(th)


LAMBDA = 8.0  # safety factor on the "rms" error scale (about 8 standard deviations)


@pytest.mark.parametrize("u_act", [0.0, 2.0 ** -9])
def test_forward_bound_holds_for_fp32_evaluation_and_is_tight(u_act):
    rng = np.random.default_rng(21)
    th = _theta(22)
    x = rng.normal(size=(3, 2, 8, 8, 8)).astype(F32).astype(np.float64)
    y, _, worst = net.forward_bound(th, x, u_act=u_act, mode="worst")
    _, _, rms = net.forward_bound(th, x, u_act=u_act, mode="rms")
    y32, _ = _forward32(th, x, act_round=net.bf16_round if u_act else None)
    err = np.abs(y32.astype(np.float64) - y)
    assert np.all(err <= worst[5]), float(np.max(err / worst[5]))
    assert np.all(err <= LAMBDA * rms[5]), float(np.max(err / rms[5]))
    # tight: far below the output scale, so one wrong entry cannot hide in it
    rel = 1e-4 if u_act == 0 else 3e-2
    assert LAMBDA * np.max(rms[5]) <= rel * np.max(np.abs(y))
    # and a planted error of one entry is caught
    bad = y32.astype(np.float64).copy()
    bad[1, 0, 3, 4, 5] += rel * np.max(np.abs(y))
    assert np.any(np.abs(bad - y) > LAMBDA * rms[5])


def test_gradient_bound_holds_for_fp32_evaluation_and_is_tight():
    rng = np.random.default_rng(23)
    th = _theta(24)
    B = 2
    x = rng.normal(size=(B, 2, 8, 8, 8)).astype(F32).astype(np.float64)
    t = rng.normal(size=(B, 8, 8, 8)).astype(F32).astype(np.float64)
    L, g, worst = net.loss_and_grad_bound(th, x, t, mode="worst")
    _, _, rms = net.loss_and_grad_bound(th, x, t, mode="rms")
    g32 = _grad32(th, x, t)
    err = np.abs(g32 - g)
    assert np.all(err <= worst), float(np.max(err / worst))
    assert np.all(err <= LAMBDA * rms), float(np.max(err / rms))
    o = 0
    for name, shp in net.SHAPES:
        n = int(np.prod(shp))
        assert LAMBDA * np.max(rms[o:o + n]) <= 1e-3 * np.max(np.abs(g[o:o + n])), name
        o += n


def test_rules_reject_unknown_mode():
    with pytest.raises(ValueError):
        net.forward_bound(_theta(1), np.zeros((1, 2, 8, 8, 8)), mode="typo")


def test_energy_gradient_bound_holds_for_fp32_evaluation():
    """The element-energy loss's gradient (the operator applied in FP32) stays
    within both the rigorous bound and lambda times the rms scale."""
    from oracle import ref
    from paper_2011_04981_gb300 import inputs

    B = 2
    mesh = inputs.box_mesh(2, 1, 1, 8, perturb=0.2, seed=6)
    Pr = ref.Problem(mesh)
    A = np.stack([ref.element_matrix(Pr.D, Pr.G[e]) for e in range(B)])
    Aabs = np.stack([ref.element_matrix(np.abs(Pr.D), np.abs(Pr.G[e])) for e in range(B)])
    rng = np.random.default_rng(25)
    th = _theta(26)
    x = rng.normal(size=(B, 2, 8, 8, 8)).astype(F32).astype(np.float64)
    t = rng.normal(size=(B, 8, 8, 8)).astype(F32).astype(np.float64)
    L, g, worst = net.energy_loss_and_grad_bound(th, x, t, A, Aabs, 8, mode="worst")
    _, _, rms = net.energy_loss_and_grad_bound(th, x, t, A, Aabs, 8, mode="rms")
    L0, g0, _ = net.energy_loss_and_grad(th, x, t, A)
    assert L == pytest.approx(L0, rel=1e-14) and np.allclose(g, g0, rtol=1e-13, atol=0)
    err = np.abs(_energy_grad32(th, x, t, A) - g)
    assert np.all(err <= worst), float(np.max(err / worst))
    o = 0
    for name, shp in net.SHAPES:
        n = int(np.prod(shp))
        if name != "b3":  # d loss / d b3 is zero up to rounding (constants are in the kernel of A)
            assert np.all(err[o:o + n] <= LAMBDA * rms[o:o + n]), (name, float(np.max(err[o:o + n] / rms[o:o + n])))
        o += n
