"""Pins for the oracle's discrete adjoint of the semi-implicit CH scheme.

The adjoint (gradients of a loss of c_N with respect to c_0, kappa and M)
is checked against (i) the tangent-linear model through the transpose
identity <w, J v> = <J^T w, v>, and (ii) central finite differences of the
forward oracle with step 1e-3.
"""
import numpy as np

from oracle import oracle as O
from paper_2507_21748_gb300 import inputs

SHAPE = (16, 16, 16)
DT, M, KAPPA, H, NSTEPS = 0.1, 1.0, 1.0, 1.0, 6


def _c0():
    return inputs.uniform_field(SHAPE, seed=11, lo=-0.4, hi=0.4, offset=0.1).astype(np.float64)


def test_transpose_identity():
    rng = np.random.default_rng(0)
    c0 = _c0()
    v = rng.standard_normal(SHAPE)
    w = rng.standard_normal(SHAPE)
    Jv = O.ch_tangent(c0, v, DT, M, KAPPA, H, NSTEPS)
    JTw, gk, gM = O.ch_adjoint(c0, w, DT, M, KAPPA, H, NSTEPS)
    lhs = float(np.sum(w * Jv))
    rhs = float(np.sum(JTw * v))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
    # parameter directions: <w, dc_N/dkappa> = gk, <w, dc_N/dM> = gM
    dk = O.ch_tangent(c0, np.zeros(SHAPE), DT, M, KAPPA, H, NSTEPS, dkappa=1.0)
    dm = O.ch_tangent(c0, np.zeros(SHAPE), DT, M, KAPPA, H, NSTEPS, dM=1.0)
    assert abs(float(np.sum(w * dk)) - gk) <= 1e-12 * max(abs(gk), 1.0)
    assert abs(float(np.sum(w * dm)) - gM) <= 1e-12 * max(abs(gM), 1.0)


def _loss(c0, kappa, M, target):
    cN = O.ch_step(c0, DT, M, kappa, H, NSTEPS, check_imag=False)
    return 0.5 * float(np.sum((cN - target) ** 2))


def test_central_differences():
    c0 = _c0()
    target = O.ch_step(c0, DT, 0.8, 1.5, H, NSTEPS)
    cN = O.ch_step(c0, DT, M, KAPPA, H, NSTEPS)
    g0, gk, gM = O.ch_adjoint(c0, cN - target, DT, M, KAPPA, H, NSTEPS)
    e = 1e-3
    fd_k = (_loss(c0, KAPPA + e, M, target) - _loss(c0, KAPPA - e, M, target)) / (2 * e)
    fd_M = (_loss(c0, KAPPA, M + e, target) - _loss(c0, KAPPA, M - e, target)) / (2 * e)
    assert abs(fd_k - gk) <= 1e-5 * abs(gk)
    assert abs(fd_M - gM) <= 1e-5 * abs(gM)
    rng = np.random.default_rng(5)
    d = rng.standard_normal(SHAPE)
    d /= np.linalg.norm(d)
    fd_c = (_loss(c0 + e * d, KAPPA, M, target) - _loss(c0 - e * d, KAPPA, M, target)) / (2 * e)
    an_c = float(np.sum(g0 * d))
    assert abs(fd_c - an_c) <= 1e-5 * abs(an_c)
