"""FP64 CPU oracle of the surrogate network (test infrastructure only).

Only tests/ and bench.py may import it. Definitions (channels-last arrays
[B, X, Y, Z, C]; weights W[t][co][ci], t = 9 (dx+1) + 3 (dy+1) + (dz+1)):

  conv(x; W, b)(v, co) = b(co) + sum_t sum_ci W[t][co][ci] x(v + off_t, ci),
  periodic in X, Y, Z;  GELU(u) = u Phi(u) (erf form).

Network (the learned surrogate of the Cahn-Hilliard step):
  h0 = conv(in; W0, b0) with in(v) = (c(v), 0, ..., 0) (16 channels)
  block k: u = conv(h; W1k, b1k), a = GELU(u), h <- h + conv(a; W2k, b2k)
  d = channel 0 of conv(h; Wp, bp)
  c_pred = c + d - mean_sample(d)
and its backward pass for the loss L = (1/(B V)) sum (c_pred - c_target)^2.
"""
import numpy as np
from scipy.special import erf

OFFS = [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)]


def shift(x, off):
    """y(v) = x(v + off), periodic over axes 1..3."""
    return np.roll(x, shift=(-off[0], -off[1], -off[2]), axis=(1, 2, 3))


def unshift(x, off):
    """adjoint of shift: y(v) = x(v - off)."""
    return np.roll(x, shift=(off[0], off[1], off[2]), axis=(1, 2, 3))


def conv(x, W, b=None):
    out = 0.0
    for t, off in enumerate(OFFS):
        out = out + shift(x, off) @ W[t].T
    return out + (0.0 if b is None else b)


def conv_dgrad(dy, W):
    """d/dx of <dy, conv(x; W)>."""
    out = 0.0
    for t, off in enumerate(OFFS):
        out = out + unshift(dy @ W[t], off)
    return out


def conv_wgrad(dy, x):
    """d/dW[t][co][ci] of <dy, conv(x; W)>."""
    co, ci = dy.shape[-1], x.shape[-1]
    dW = np.zeros((27, co, ci))
    dyf = dy.reshape(-1, co)
    for t, off in enumerate(OFFS):
        dW[t] = dyf.T @ shift(x, off).reshape(-1, ci)
    return dW


def gelu(u):
    return 0.5 * u * (1.0 + erf(u / np.sqrt(2.0)))


def gelu_grad(u):
    return 0.5 * (1.0 + erf(u / np.sqrt(2.0))) + u * np.exp(-0.5 * u * u) / np.sqrt(2.0 * np.pi)


def field_to_act(c, C=16):
    a = np.zeros(c.shape + (C,))
    a[..., 0] = c
    return a


def forward(params, c):
    """params: dict W0, b0, blocks [(W1, b1, W2, b2)], Wp, bp. c: [B, X, Y, Z]."""
    cache = {}
    a_in = field_to_act(np.asarray(c, dtype=np.float64))
    h = conv(a_in, params["W0"], params["b0"])
    cache["a_in"], hs, us, as_ = a_in, [h], [], []
    for (W1, b1, W2, b2) in params["blocks"]:
        u = conv(h, W1, b1)
        a = gelu(u)
        h = h + conv(a, W2, b2)
        us.append(u)
        as_.append(a)
        hs.append(h)
    d = conv(h, params["Wp"], params["bp"])[..., 0]
    d0 = d - d.mean(axis=(1, 2, 3), keepdims=True)
    cache.update(hs=hs, us=us, as_=as_)
    return np.asarray(c, dtype=np.float64) + d0, cache


def loss_and_grads(params, c, target):
    B = c.shape[0]
    V = int(np.prod(c.shape[1:]))
    pred, cache = forward(params, c)
    L = float(np.sum((pred - target) ** 2)) / (B * V)
    dpred = 2.0 * (pred - target) / (B * V)
    gd = dpred - dpred.mean(axis=(1, 2, 3), keepdims=True)
    g = {}
    dyp = field_to_act(gd)
    hs, us, as_ = cache["hs"], cache["us"], cache["as_"]
    g["Wp"] = conv_wgrad(dyp, hs[-1])
    g["bp"] = dyp.sum(axis=(0, 1, 2, 3))
    dh = conv_dgrad(dyp, params["Wp"])
    g["blocks"] = [None] * len(params["blocks"])
    for k in range(len(params["blocks"]) - 1, -1, -1):
        W1, b1, W2, b2 = params["blocks"][k]
        dW2 = conv_wgrad(dh, as_[k])
        db2 = dh.sum(axis=(0, 1, 2, 3))
        du = conv_dgrad(dh, W2) * gelu_grad(us[k])
        dW1 = conv_wgrad(du, hs[k])
        db1 = du.sum(axis=(0, 1, 2, 3))
        dh = dh + conv_dgrad(du, W1)
        g["blocks"][k] = (dW1, db1, dW2, db2)
    g["W0"] = conv_wgrad(dh, cache["a_in"])
    g["b0"] = dh.sum(axis=(0, 1, 2, 3))
    return L, pred, g
