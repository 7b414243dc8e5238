"""Pins for the oracle's Cahn-Hilliard step (test infrastructure).

Each test checks the oracle against something other than itself: a closed
form of the scheme, an invariant, or a property of the PDE that the scheme
(Appendix "Semi-implicit timestepping", update with S = -M kappa |k|^4)
must keep.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_21748_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_increment_form_equals_update_form():
    """The appendix's increment form c + F^-1{dt/(1 - dt S) F{rhs}} with the
    spectral rhs equals (c_hat - dt M k^2 g_hat)/(1 + dt M kappa k^4)."""
    c = inputs.uniform_field((16, 12, 10), seed=5, lo=-0.5, hi=0.5)
    a = O.ch_step(c, 0.1, 0.7, 1.3, h=0.9, nsteps=3)
    b = O.ch_step_increment(c, 0.1, 0.7, 1.3, h=0.9, nsteps=3)
    assert np.abs(a - b).max() < 1e-13


def test_zero_mobility_is_identity():
    c = inputs.uniform_field((12, 8, 10), seed=1, lo=-1, hi=1)
    out = O.ch_step(c, 0.1, 0.0, 1.0, nsteps=4)
    assert np.abs(out - c).max() < 1e-14


def test_constant_field_is_fixed_point():
    c = np.full((8, 10, 12), 0.37, dtype=np.float32)
    out = O.ch_step(c, 0.5, 1.0, 2.0, nsteps=3)
    assert np.abs(out - np.float64(np.float32(0.37))).max() < 1e-15


def test_dc_independent_of_kappa_and_exact_mass():
    c = inputs.uniform_field((16, 16, 16), seed=2, offset=0.3)
    m0 = O.mass(c)
    l1 = np.abs(c.astype(np.float64)).sum()
    for kappa in (0.5, 1.0, 3.0):
        out = O.ch_step(c, 0.1, 1.0, kappa, nsteps=10)
        assert abs(O.mass(out) - m0) / l1 < 1e-13


@pytest.mark.parametrize("h", [1.0, 0.8])
@pytest.mark.parametrize("mvec,A", [((3, 0, 0), 0.8), ((1, 2, 0), 0.5), ((2, 1, 1), 1.2)])
def test_single_mode_closed_form(mvec, A, h):
    """c = A cos(k1.x). Since cos^3 = (3 cos + cos 3)/4, g = (3A^3/4 - A) cos + (A^3/4) cos 3,
    so one step gives exactly alpha cos(k1.x) + beta cos(3 k1.x) with
    alpha = (A - dt M k1^2 (3A^3/4 - A)) / (1 + dt M kappa k1^4),
    beta  = -dt M 9 k1^2 (A^3/4) / (1 + dt M kappa 81 k1^4),
    k1^2 = sum_d (2 pi m_d / (N h))^2. At h = 0.8 the wave numbers grow by 1/h,
    which pins the voxel edge's scaling of the symbols."""
    N = 32
    dt, M, kappa = 0.2, 0.9, 1.1
    x = np.indices((N, N, N)).astype(np.float64)
    theta = 2 * np.pi * sum(mvec[d] * x[d] for d in range(3)) / N
    c = A * np.cos(theta)
    k1sq = sum((2 * np.pi * m / (N * h)) ** 2 for m in mvec)
    alpha = (A - dt * M * k1sq * (0.75 * A ** 3 - A)) / (1 + dt * M * kappa * k1sq ** 2)
    beta = -dt * M * 9 * k1sq * (A ** 3 / 4) / (1 + dt * M * kappa * 81 * k1sq ** 2)
    expect = alpha * np.cos(theta) + beta * np.cos(3 * theta)
    got = O.ch_step(c, dt, M, kappa, h, 1)
    assert np.abs(got - expect).max() < 1e-13


def _golden_growth():
    rows = []
    with open(os.path.join(GOLDEN, "growth_factor_64.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                m, G = line.split()
                rows.append((int(m), float(G)))
    return rows


def test_linearised_growth_matches_golden():
    """A small mode on cbar = 0 grows or decays by the closed-form G(k) per step
    (self-interaction changes G only at O(eps^2)). Each mode runs on its own so
    that cubic cross terms of growing modes cannot feed a decaying one."""
    N, eps, nsteps = 64, 1e-6, 50
    x = np.arange(N, dtype=np.float64)
    for m, G in _golden_growth():
        line = eps * np.cos(2 * np.pi * m * x / N)
        c = np.broadcast_to(line[:, None, None], (N, 4, 4)).copy()
        out = O.ch_step(c, 0.1, 1.0, 1.0, 1.0, nsteps, check_imag=False)
        s0 = O.fftn(c)[m, 0, 0].real
        s1 = O.fftn(out)[m, 0, 0].real
        rate = (s1 / s0) ** (1.0 / nsteps)
        assert abs(rate - G) < 6e-9, (m, rate, G)


def test_linearised_growth_offcritical():
    """Same at cbar = 0.3 (the off-critical mixture), against the closed form."""
    N, eps, nsteps, cbar = 64, 1e-7, 50, 0.3
    dt, M, kappa = 0.1, 1.0, 1.0
    x = np.arange(N, dtype=np.float64)
    ms = [2, 7, 13]
    line = cbar + sum(eps * np.cos(2 * np.pi * m * x / N) for m in ms)
    c = np.broadcast_to(line[:, None, None], (N, 4, 4)).copy()
    out = O.ch_step(c, dt, M, kappa, 1.0, nsteps, check_imag=False)
    s0 = O.fftn(c)[:, 0, 0]
    s1 = O.fftn(out)[:, 0, 0]
    for m in ms:
        k2 = (2 * np.pi * m / N) ** 2
        G = (1 - dt * M * k2 * (3 * cbar ** 2 - 1)) / (1 + dt * M * kappa * k2 * k2)
        rate = (s1[m].real / s0[m].real) ** (1.0 / nsteps)
        assert abs(rate - G) < 1e-8 * G, (m, rate, G)


@pytest.mark.parametrize("offset", [0.0, 0.3])
def test_energy_monotone(offset):
    """The semi-implicit scheme decreases the Ginzburg-Landau energy at dt = 0.1."""
    c = inputs.uniform_field((32, 32, 32), seed=7, offset=offset)
    out, E = O.ch_step(c, 0.1, 1.0, 1.0, 1.0, 200, energies=True)
    assert np.all(np.diff(E) <= 1e-12 * np.abs(E[:-1]))
    assert E[-1] < E[0]


@pytest.mark.parametrize("h", [1.0, 0.8])
@pytest.mark.parametrize("m", [(3, 0, 0), (1, 2, 3)])
def test_energy_closed_form_single_mode(m, h):
    """E of A cos(k.x) on an n-grid of edge h: the bulk term is h^3 sum (c^2-1)^2/4 =
    h^3 V (3A^4/8 - A^2 + 1)/4 (means of cos^2 and cos^4 over whole periods: 1/2, 3/8),
    and the gradient term h^3 (kappa/2) sum |grad c|^2 = h^3 (kappa/2) |k|^2 A^2 V/2 with
    |k|^2 = sum_d (2 pi m_d / (n_d h))^2. At h = 0.8 the bulk term scales by h^3 and the
    gradient term by h, which pins both factors."""
    n, A, kappa = (16, 12, 20), 0.4, 1.5
    X, Y, Z = np.meshgrid(*[np.arange(nd) for nd in n], indexing="ij")
    c = A * np.cos(2 * np.pi * (m[0] * X / n[0] + m[1] * Y / n[1] + m[2] * Z / n[2]))
    V = n[0] * n[1] * n[2]
    k2 = sum((2 * np.pi * m[d] / (n[d] * h)) ** 2 for d in range(3))
    bulk = h ** 3 * V * (A ** 4 * 3 / 8 - A ** 2 + 1) / 4
    grad = h ** 3 * 0.5 * kappa * k2 * A ** 2 * V / 2
    assert abs(O.energy(c, kappa, h) - (bulk + grad)) < 1e-10 * (bulk + grad)


def test_first_order_in_dt():
    """IMEX Euler is first order: successive differences halve with dt."""
    shape = (32, 32, 32)
    c0 = inputs.mode_field(shape, [(0.1, (1, 0, 0), 0.3), (0.1, (0, 2, 1), 1.1), (0.1, (1, 1, 2), 2.0)])
    T = 2.0
    dts = [0.1, 0.05, 0.025, 0.0125, 0.00625]
    sols = [O.ch_step(c0, dt, 1.0, 1.0, 1.0, int(round(T / dt)), check_imag=False) for dt in dts]
    diffs = [np.sqrt(np.mean((sols[i] - sols[i + 1]) ** 2)) for i in range(len(sols) - 1)]
    orders = [math.log2(diffs[i] / diffs[i + 1]) for i in range(len(diffs) - 1)]
    assert all(0.9 <= p <= 1.1 for p in orders), orders


def test_step_modes_matches_full_step():
    """Mode-by-mode evaluation (direct sums) equals the full FFT step."""
    c = inputs.uniform_field((16, 12, 10), seed=3, offset=0.3)
    dt, M, kappa, h = 0.1, 1.0, 1.0, 1.0
    full = O.fftn(O.ch_step(c, dt, M, kappa, h, 1))
    modes = np.array([[0, 0, 0], [1, 0, 0], [5, 7, 3], [15, 11, 9], [8, 6, 5], [2, 3, 1]])
    got = O.step_modes(c, modes, dt, M, kappa, h)
    for i, (a, b, d) in enumerate(modes):
        assert abs(got[i] - full[a, b, d]) < 1e-11


def test_block_step_of_one_step_is_the_scheme():
    """The block propagator with n = 1 is one step of the scheme (the split
    g = g(cbar) + g'(cbar) d + N(d) is exact and g(cbar) only feeds k = 0)."""
    c = inputs.uniform_field((16, 12, 10), seed=5, offset=0.2, lo=-0.6, hi=0.6)
    for h in (1.0, 0.8):
        a = O.ch_step(c, 0.1, 0.7, 1.3, h, 1)
        b = O.ch_block_step(c, 0.1, 0.7, 1.3, h, 1)
        assert np.abs(a - b).max() < 1e-13


def test_block_step_linear_regime_and_cosine_closed_form():
    """A tiny mode on cbar follows L(k)^n exactly up to O(eps^2); a cosine mode's
    block has the closed form from N = d^2 (3 cbar + d) of d = A cos(t):
    3 cbar A^2/2 (1 + cos 2t) + (3A^3/4) cos t + (A^3/4) cos 3t, each mode of N
    multiplied by B S_n with S_n = sum_{j<n} L^j."""
    N, dt, M, kappa, cbar, n = 32, 0.1, 0.9, 1.1, 0.25, 10
    x = np.indices((N, N, N)).astype(np.float64)
    mvec = (2, 1, 0)
    theta = 2 * np.pi * sum(mvec[d] * x[d] for d in range(3)) / N

    def LBS(mult):
        k2 = sum((2 * np.pi * mult * m / N) ** 2 for m in mvec)
        D = 1 + dt * M * kappa * k2 * k2
        L = (1 - dt * M * k2 * (3 * cbar * cbar - 1)) / D
        return L, -dt * M * k2 / D, sum(L ** j for j in range(n))

    A = 0.3
    c = cbar + A * np.cos(theta)
    (L1, B1, S1), (L2, B2, S2), (L3, B3, S3) = LBS(1), LBS(2), LBS(3)
    expect = (cbar + (L1 ** n * A + B1 * S1 * 0.75 * A ** 3) * np.cos(theta)
              + B2 * S2 * 1.5 * cbar * A * A * np.cos(2 * theta) + B3 * S3 * 0.25 * A ** 3 * np.cos(3 * theta))
    got = O.ch_block_step(c, dt, M, kappa, 1.0, n)
    assert np.abs(got - expect).max() < 1e-13
    eps = 1e-7
    c = cbar + eps * np.cos(theta)
    got = O.ch_block_step(c, dt, M, kappa, 1.0, n) - cbar
    assert np.abs(got - L1 ** n * eps * np.cos(theta)).max() < 20 * eps * eps  # the O(eps^2) of N
