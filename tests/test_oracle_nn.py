"""Pins for the oracle of the surrogate network (test infrastructure).

The periodic convolution is checked against a brute-force loop written from
its definition, its data and weight gradients through transpose identities,
GELU's derivative and the whole network's gradients by central differences.
"""
import numpy as np

from oracle import nn as N


def brute_conv(x, W, b):
    B, X, Y, Z, C = x.shape
    out = np.zeros((B, X, Y, Z, W.shape[1]))
    for bb in range(B):
        for i in range(X):
            for j in range(Y):
                for k in range(Z):
                    acc = b.copy()
                    for t, (dx, dy, dz) in enumerate(N.OFFS):
                        acc = acc + W[t] @ x[bb, (i + dx) % X, (j + dy) % Y, (k + dz) % Z]
                    out[bb, i, j, k] = acc
    return out


def test_conv_vs_bruteforce():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 4, 5, 3))
    W = rng.standard_normal((27, 4, 3))
    b = rng.standard_normal(4)
    assert np.abs(N.conv(x, W, b) - brute_conv(x, W, b)).max() < 1e-12


def test_conv_gradients_transpose_identities():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 4, 3, 5, 3))
    W = rng.standard_normal((27, 4, 3))
    dy = rng.standard_normal((2, 4, 3, 5, 4))
    lhs = np.sum(dy * N.conv(x, W))
    assert abs(lhs - np.sum(N.conv_dgrad(dy, W) * x)) < 1e-10 * abs(lhs)
    assert abs(lhs - np.sum(N.conv_wgrad(dy, x) * W)) < 1e-10 * abs(lhs)


def test_gelu_grad_central_difference():
    u = np.linspace(-4, 4, 81)
    e = 1e-6
    fd = (N.gelu(u + e) - N.gelu(u - e)) / (2 * e)
    assert np.abs(fd - N.gelu_grad(u)).max() < 1e-8
    # closed values: GELU(0) = 0, GELU'(0) = 1/2
    assert N.gelu(np.array(0.0)) == 0.0 and abs(N.gelu_grad(np.array(0.0)) - 0.5) < 1e-15


def small_params(rng, C=4, nb=2):
    def w(co, ci, s):
        return rng.standard_normal((27, co, ci)) * s
    return {"W0": w(C, 16, 0.3), "b0": rng.standard_normal(C) * 0.1,
            "blocks": [(w(C, C, 0.2), rng.standard_normal(C) * 0.1, w(C, C, 0.2), rng.standard_normal(C) * 0.1)
                       for _ in range(nb)],
            "Wp": w(16, C, 0.2), "bp": rng.standard_normal(16) * 0.1}


def test_network_gradients_central_differences():
    rng = np.random.default_rng(2)
    p = small_params(rng)
    c = rng.standard_normal((2, 4, 4, 4)) * 0.3
    tgt = rng.standard_normal((2, 4, 4, 4)) * 0.3
    L, pred, g = N.loss_and_grads(p, c, tgt)
    # mass: the correction is zero-mean per sample
    assert np.abs((pred - c).mean(axis=(1, 2, 3))).max() < 1e-14 * np.abs(pred - c).max()
    e = 1e-5
    probes = [("W0", (3, 1, 0)), ("b0", (2,)), ("Wp", (13, 0, 2)), ("bp", (0,))]
    for name, idx in probes:
        q = {k: v for k, v in p.items()}
        a = p[name].copy()
        a[idx] += e
        q[name] = a
        Lp = N.loss_and_grads(q, c, tgt)[0]
        a = p[name].copy()
        a[idx] -= e
        q[name] = a
        Lm = N.loss_and_grads(q, c, tgt)[0]
        fd = (Lp - Lm) / (2 * e)
        assert abs(fd - g[name][idx]) < 1e-6 * max(1e-3, abs(fd)), (name, fd, g[name][idx])
    for k, j, idx in [(0, 0, (5, 1, 2)), (1, 2, (20, 3, 0)), (1, 1, (2,))]:
        blocks = [list(b) for b in p["blocks"]]
        base = blocks[k][j].copy()
        blocks[k][j] = base.copy(); blocks[k][j][idx] += e
        Lp = N.loss_and_grads(dict(p, blocks=[tuple(b) for b in blocks]), c, tgt)[0]
        blocks[k][j] = base.copy(); blocks[k][j][idx] -= e
        Lm = N.loss_and_grads(dict(p, blocks=[tuple(b) for b in blocks]), c, tgt)[0]
        fd = (Lp - Lm) / (2 * e)
        assert abs(fd - g["blocks"][k][j][idx]) < 1e-6 * max(1e-3, abs(fd))
