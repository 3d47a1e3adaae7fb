"""Oracle for the learned element preconditioner (plain numpy, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has no learned component; this is the per-element network of the
learned-preconditioner extension, written out from its definition:

* input  x[b, c, k, j, i]  (c = 0: residual, c = 1: Jacobi-scaled residual, each
  divided by its element RMS), an nx^3 block per element;
* conv(x; W, bias)[o] = bias[o] + sum_c sum_{taps t} W[o, c, t] x[c, p + t] with
  t over the 27 offsets {-1,0,1}^3 and zero outside the element ("same" padding
  inside each element), tap index t = (dk+1)*9 + (dj+1)*3 + (di+1);
* layers: h1 = conv(x; W1, b1), a1 = gelu(h1); h2 = conv(a1; W2, b2),
  a2 = gelu(h2); y = conv(a2; W3, b3), with 16 hidden channels;
* gelu(v) = v * Phi(v) = 0.5 v (1 + erf(v / sqrt 2));
* loss per sample ||y - t||^2 / ||t||^2, averaged over the batch.

Parameters are one flat vector: W1 [16,2,27], b1 [16], W2 [16,16,27], b2 [16],
W3 [1,16,27], b3 [1] (8241 values).  The backward pass is the chain rule
written out layer by layer.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

CIN, CH = 2, 16
SHAPES = [("W1", (CH, CIN, 27)), ("b1", (CH,)), ("W2", (CH, CH, 27)), ("b2", (CH,)), ("W3", (1, CH, 27)),
          ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)

TAPS = [(dk, dj, di) for dk in (-1, 0, 1) for dj in (-1, 0, 1) for di in (-1, 0, 1)]


def unpack(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def shift(x, dk, dj, di):
    """s[..., k, j, i] = x[..., k+dk, j+dj, i+di], zero outside the block."""
    n = x.shape[-1]
    out = np.zeros_like(x)
    ks = slice(max(0, -dk), min(n, n - dk))
    js = slice(max(0, -dj), min(n, n - dj))
    is_ = slice(max(0, -di), min(n, n - di))
    kt = slice(max(0, dk), min(n, n + dk))
    jt = slice(max(0, dj), min(n, n + dj))
    it = slice(max(0, di), min(n, n + di))
    out[..., ks, js, is_] = x[..., kt, jt, it]
    return out


def conv(x, W, b):
    """x [B, Cin, n, n, n], W [Cout, Cin, 27], b [Cout] -> [B, Cout, n, n, n]."""
    y = np.zeros((x.shape[0], W.shape[0]) + x.shape[2:])
    for t, (dk, dj, di) in enumerate(TAPS):
        y += np.einsum("oc,bckji->bokji", W[:, :, t], shift(x, dk, dj, di))
    return y + b[None, :, None, None, None]


def conv_input_grad(dy, W):
    """d/dx of sum(dy * conv(x)): sum over taps of W^T applied to dy shifted the other way."""
    dx = np.zeros((dy.shape[0], W.shape[1]) + dy.shape[2:])
    for t, (dk, dj, di) in enumerate(TAPS):
        dx += shift(np.einsum("oc,bokji->bckji", W[:, :, t], dy), -dk, -dj, -di)
    return dx


def conv_weight_grad(dy, x):
    """d/dW[o,c,t] of sum(dy * conv(x)) = sum_{b,p} dy[b,o,p] x[b,c,p+t]."""
    dW = np.zeros((dy.shape[1], x.shape[1], 27))
    for t, (dk, dj, di) in enumerate(TAPS):
        dW[:, :, t] = np.einsum("bokji,bckji->oc", dy, shift(x, dk, dj, di))
    return dW


def gelu(v):
    return 0.5 * v * (1.0 + erf(v / math.sqrt(2.0)))


def gelu_grad(v):
    return 0.5 * (1.0 + erf(v / math.sqrt(2.0))) + v * np.exp(-0.5 * v * v) / math.sqrt(2.0 * math.pi)


def bf16_round(v):
    """Round to the nearest BF16 value (ties to even), via FP32: the FP32 bit
    pattern plus 0x7FFF plus the lowest kept bit, truncated to the top 16 bits
    (finite values)."""
    f = np.asarray(v, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, x, keep=False, act_round=None):
    """act_round (optional): applied to the network input and to both hidden
    activations before the convolution that reads them (the reduced-precision
    inference form)."""
    P = unpack(theta)
    rnd = act_round if act_round is not None else (lambda v: v)
    x = rnd(x)
    h1 = conv(x, P["W1"], P["b1"])
    a1 = rnd(gelu(h1))
    h2 = conv(a1, P["W2"], P["b2"])
    a2 = rnd(gelu(h2))
    y = conv(a2, P["W3"], P["b3"])
    if keep:
        return y, (x, h1, a1, h2, a2)
    return y


def loss(theta, x, t):
    y = forward(theta, x)[:, 0]
    num = np.sum((y - t) ** 2, axis=(1, 2, 3))
    den = np.sum(t ** 2, axis=(1, 2, 3))
    return float(np.mean(num / den))


def backward(theta, cache, dy):
    """Gradients of sum(dy * y) with respect to theta and to the input."""
    P = unpack(theta)
    x0, h1, a1, h2, a2 = cache
    g = {}
    g["W3"] = conv_weight_grad(dy, a2)
    g["b3"] = dy.sum(axis=(0, 2, 3, 4))
    dh2 = conv_input_grad(dy, P["W3"]) * gelu_grad(h2)
    g["W2"] = conv_weight_grad(dh2, a1)
    g["b2"] = dh2.sum(axis=(0, 2, 3, 4))
    dh1 = conv_input_grad(dh2, P["W2"]) * gelu_grad(h1)
    g["W1"] = conv_weight_grad(dh1, x0)
    g["b1"] = dh1.sum(axis=(0, 2, 3, 4))
    dx = conv_input_grad(dh1, P["W1"])
    return pack(g), dx


def loss_and_grad(theta, x, t):
    """Loss and its gradient with respect to theta (and to the input x)."""
    y, cache = forward(theta, x, keep=True)
    B = x.shape[0]
    den = np.sum(t ** 2, axis=(1, 2, 3))
    r = y[:, 0] - t
    L = float(np.mean(np.sum(r ** 2, axis=(1, 2, 3)) / den))
    dy = (2.0 / B) * (r / den[:, None, None, None])[:, None]
    g, dx = backward(theta, cache, dy)
    return L, g, dx


def energy_loss(theta, x, t, A):
    """mean_b (y_b - t_b)^T A_b (y_b - t_b) / t_b^T A_b t_b with A [B, n^3, n^3] (element matrices)."""
    B = x.shape[0]
    y = forward(theta, x)[:, 0].reshape(B, -1)
    tt = t.reshape(B, -1)
    d = y - tt
    num = np.einsum("bp,bpq,bq->b", d, A, d)
    den = np.einsum("bp,bpq,bq->b", tt, A, tt)
    return float(np.mean(num / den))


def energy_loss_and_grad(theta, x, t, A):
    B = x.shape[0]
    y, cache = forward(theta, x, keep=True)
    yf = y[:, 0].reshape(B, -1)
    tt = t.reshape(B, -1)
    d = yf - tt
    Ad = np.einsum("bpq,bq->bp", A, d)
    den = np.einsum("bp,bpq,bq->b", tt, A, tt)
    L = float(np.mean(np.sum(d * Ad, axis=1) / den))
    dy = ((2.0 / B) * Ad / den[:, None]).reshape(y.shape)
    g, dx = backward(theta, cache, dy)
    return L, g, dx


def adam(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, 2015) from step count t >= 1."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def element_inputs(r, jr):
    """Per-element RMS normalisation of the two input channels; returns (x, s_r, s_j)."""
    sr = np.sqrt(np.mean(r * r, axis=1))
    sj = np.sqrt(np.mean(jr * jr, axis=1))
    x = np.stack([np.where(sr[:, None] > 0, r / np.where(sr > 0, sr, 1)[:, None], 0.0),
                  np.where(sj[:, None] > 0, jr / np.where(sj > 0, sj, 1)[:, None], 0.0)], axis=1)
    return x, sr, sj


# ---------------------------------------------------------------------------
# Componentwise rounding-error bounds of a reduced-precision evaluation.
#
# The GPU kernels evaluate the network in FP32 (and, in the tensor-core form,
# round the input and the hidden activations to BF16 first).  Every rounding
# follows the standard model fl(a op b) = (a op b)(1 + d), |d| <= u, and each
# output, activation and gradient entry gets its own bound, propagated through
# the layers to first order.  Two modes:
#
# * "worst": a sum of n terms is off by at most gamma_n = n u / (1 - n u) times
#   the sum of the terms' absolute values, and an input error bound e_i reaches
#   a linear output as sum_i |W_i| e_i (Higham, "Accuracy and Stability of
#   Numerical Algorithms", Sec. 3.1).  Rigorous for any summation order, but it
#   compounds the worst case of every layer, and through three 16-channel
#   3x3x3 layers it overstates the error by orders of magnitude.
# * "rms": roundings are independent and of mean zero (the model of Higham and
#   Mary, "A new approach to probabilistic rounding error analysis", SIAM J.
#   Sci. Comput. 2019): the sum's own error scales as sqrt(n) u times the sum
#   of absolute values, and errors carried in from the inputs combine as
#   sqrt(sum_i W_i^2 e_i^2); independent contributions add in quadrature.  The
#   result is an error scale; a test multiplies it by a safety factor lambda.
# ---------------------------------------------------------------------------

U32 = 2.0 ** -24
GELU_LIP = 1.1290      # max |gelu'(v)|, reached at v = sqrt(2)
GELU2_LIP = 0.7979     # max |gelu''(v)| = 2 phi(0)
GELU_ABS = 8 * U32     # FP32 gelu: relative error in |gelu| plus absolute error in |v| (erf near -1)
GELUP_ABS = 16 * U32   # FP32 gelu': absolute error (it is O(1))


def gamma(n, u=U32):
    return n * u / (1.0 - n * u)


class _Rules:
    """How errors combine in one mode (see above)."""

    def __init__(self, mode, u):
        if mode not in ("worst", "rms"):
            raise ValueError(mode)
        self.worst, self.u = mode == "worst", u

    def sum_err(self, n):
        """Factor on the sum of absolute values for a sum of n rounded terms."""
        return gamma(n, self.u) if self.worst else math.sqrt(n) * self.u

    def add(self, *parts):
        if self.worst:
            return sum(parts)
        return np.sqrt(sum(np.asarray(p) ** 2 for p in parts))

    def lin(self, f, e, W):
        """Error carried through a linear map f(input, weights) from input errors e."""
        return f(e, np.abs(W)) if self.worst else np.sqrt(f(e * e, W * W))

    def bil(self, f, e1, a2, a1, e2):
        """Error of f(v1, v2) (bilinear, e.g. a weight gradient) from errors e1, e2 of v1, v2."""
        if self.worst:
            return f(e1, np.abs(a2)) + f(np.abs(a1), e2)
        return np.sqrt(f(e1 * e1, a2 * a2) + f(a1 * a1, e2 * e2))


def _conv_nb(x, W):
    return conv(x, W, np.zeros(W.shape[0]))


def forward_bound(theta, x, u_act=0.0, u=U32, mode="worst"):
    """(y, cache, bounds): the FP64 network on x and, per output, the error bound
    (mode "worst") or error scale (mode "rms") of an evaluation with unit
    roundoff u in every sum and with the input and both hidden activations
    rounded to a unit roundoff u_act (0 = no rounding) before the convolution
    that reads them.  bounds = (dx0, dh1, da1, dh2, da2, dy), each an array of
    the matching activation's shape."""
    R = _Rules(mode, u)
    P = unpack(theta)
    y, cache = forward(theta, x, keep=True)
    x0, h1, a1, h2, a2 = cache
    dx0 = u_act * np.abs(x0)

    def layer(a, da, W, b, cin):
        absum = _conv_nb(np.abs(a) + da, np.abs(W)) + np.abs(b)[None, :, None, None, None]
        return R.add(R.lin(_conv_nb, da, W), R.sum_err(27 * cin + 1) * absum)

    def act(h, a, dh):
        da = R.add(GELU_LIP * dh, GELU_ABS * (np.abs(a) + np.abs(h)))
        return R.add(da, u_act * (np.abs(a) + da))

    dh1 = layer(x0, dx0, P["W1"], P["b1"], CIN)
    da1 = act(h1, a1, dh1)
    dh2 = layer(a1, da1, P["W2"], P["b2"], CH)
    da2 = act(h2, a2, dh2)
    dy = layer(a2, da2, P["W3"], P["b3"], CH)
    return y, cache, (dx0, dh1, da1, dh2, da2, dy)


def _backward_bound(theta, cache, fb, dy, ddy, B, R):
    """Per-parameter bound (or scale) of the gradient of sum(dy * y) evaluated
    with roundoff R.u from a forward whose errors are fb (forward_bound) and an
    output gradient dy known to within ddy.  Weight-gradient sums run over the
    points of a sample and then over the batch: 512 + B terms."""
    P = unpack(theta)
    x0, h1, a1, h2, a2 = cache
    _, dh1e, da1e, dh2e, da2e, _ = fb
    nsum = x0.shape[2] * x0.shape[3] * x0.shape[4] + B
    g = {}

    def wgrad(dh, ddh, a, da):
        absum = conv_weight_grad(np.abs(dh), np.abs(a) + da)
        return R.add(R.bil(conv_weight_grad, ddh, a, dh, da), R.sum_err(nsum) * absum)

    def bgrad(dh, ddh):
        s = (lambda v: v.sum(axis=(0, 2, 3, 4)))
        carried = s(ddh) if R.worst else np.sqrt(s(ddh * ddh))
        return R.add(carried, R.sum_err(nsum) * s(np.abs(dh)))

    def through(dh_out, ddh_out, W, cout, h, dhe):
        v = conv_input_grad(dh_out, W)
        dv = R.add(R.lin(conv_input_grad, ddh_out, W),
                   R.sum_err(27 * cout) * conv_input_grad(np.abs(dh_out), np.abs(W)))
        gp = gelu_grad(h)
        dh = v * gp
        ddh = R.add(dv * np.abs(gp), (np.abs(v) + dv) * (GELU2_LIP * dhe + GELUP_ABS), R.u * np.abs(dh))
        return dh, ddh

    g["W3"] = wgrad(dy, ddy, a2, da2e)
    g["b3"] = bgrad(dy, ddy)
    dh2, ddh2 = through(dy, ddy, P["W3"], 1, h2, dh2e)
    g["W2"] = wgrad(dh2, ddh2, a1, da1e)
    g["b2"] = bgrad(dh2, ddh2)
    dh1, ddh1 = through(dh2, ddh2, P["W2"], CH, h1, dh1e)
    g["W1"] = wgrad(dh1, ddh1, x0, 0.0 * x0)
    g["b1"] = bgrad(dh1, ddh1)
    return pack(g)


def loss_and_grad_bound(theta, x, t, u=U32, mode="worst"):
    """(L, grad, bound): loss_and_grad plus a per-parameter error bound (or
    scale, mode "rms") of an FP32 evaluation: forward, loss, backward and the
    sum over the batch."""
    R = _Rules(mode, u)
    B = x.shape[0]
    y, cache, fb = forward_bound(theta, x, 0.0, u, mode)
    n = t[0].size
    den = np.sum(t ** 2, axis=(1, 2, 3))
    r = y[:, 0] - t
    L = float(np.mean(np.sum(r ** 2, axis=(1, 2, 3)) / den))
    dy = (2.0 / B) * (r / den[:, None, None, None])[:, None]
    dr = R.add(fb[5][:, 0], u * np.abs(r))
    ddy = R.add((2.0 / B) * (R.add(dr, R.sum_err(n) * np.abs(r)) / den[:, None, None, None])[:, None],
                3 * u * np.abs(dy))
    g, _ = backward(theta, cache, dy)
    return L, g, _backward_bound(theta, cache, fb, dy, ddy, B, R)


def energy_loss_and_grad_bound(theta, x, t, A, Aabs, nx, u=U32, mode="worst"):
    """(L, grad, bound) of the element-energy loss, with A d and A t formed by a
    reduced-precision operator whose componentwise error is at most
    4 (u + (2 nx + 3) u) Aabs |v| (Aabs = the element matrix of |D| and |G|)."""
    R = _Rules(mode, u)
    B = x.shape[0]
    y, cache, fb = forward_bound(theta, x, 0.0, u, mode)
    yf = y[:, 0].reshape(B, -1)
    tt = t.reshape(B, -1)
    d = yf - tt
    Ad = np.einsum("bpq,bq->bp", A, d)
    den = np.einsum("bp,bpq,bq->b", tt, A, tt)
    L = float(np.mean(np.sum(d * Ad, axis=1) / den))
    dy = ((2.0 / B) * Ad / den[:, None]).reshape(y.shape)
    g, _ = backward(theta, cache, dy)
    cax = 4 * (u + (2 * nx + 3) * u)
    dd = R.add(fb[5][:, 0].reshape(B, -1), u * np.abs(d))
    mv = (lambda e, M: np.einsum("bpq,bq->bp", M, e))
    dAd = R.add(R.lin(mv, dd, Aabs) if not R.worst else mv(dd, Aabs), cax * mv(np.abs(d) + dd, Aabs))
    At_abs = mv(np.abs(tt), Aabs)
    dden = (cax + R.sum_err(tt.shape[1]) * (1 + cax)) * np.sum(np.abs(tt) * At_abs, axis=1)
    ddy = R.add((2.0 / B) * dAd / den[:, None], (2.0 / B) * np.abs(Ad) * dden[:, None] / den[:, None] ** 2,
                3 * u * np.abs(dy.reshape(B, -1)))
    return L, g, _backward_bound(theta, cache, fb, dy, ddy.reshape(y.shape), B, R)
