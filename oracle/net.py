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
