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
