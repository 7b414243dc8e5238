"""Pins for the oracle's Allen-Cahn step (test infrastructure): Eq. (allen-cahn)
with the semi-implicit recipe of "Semi-implicit timestepping", S = -L kappa |k|^2.

Each pin checks the oracle against something other than itself: a scalar
recurrence, a closed form built from the cos^3 identity, the increment form,
the linearised growth factor, energy decay and first-order convergence."""
import numpy as np
import pytest

from oracle import oracle as O


def test_constant_field_follows_the_scalar_recurrence():
    # a uniform field has only the k = 0 mode, where the denominator is 1:
    # c' = c - dt L (c^3 - c), the explicit Euler map of c_t = -L (c^3 - c)
    dt, L, kappa = 0.1, 1.3, 0.7
    c0 = 0.37
    c = np.full((6, 4, 8), c0)
    got = O.ac_step(c, dt, L, kappa, nsteps=12)
    ref = c0
    for _ in range(12):
        ref = ref - dt * L * (ref ** 3 - ref)
    assert np.abs(got - ref).max() < 1e-14
    # and it relaxes towards the well at +1
    assert abs(ref - 1.0) < abs(c0 - 1.0)


def test_zero_mobility_is_identity_and_wells_are_fixed_points():
    rng = np.random.default_rng(0)
    c = rng.uniform(-0.5, 0.5, (8, 6, 4))
    assert np.abs(O.ac_step(c, 0.1, 0.0, 1.0, nsteps=3) - c).max() < 1e-14  # FFT round trip only
    for w in (-1.0, 0.0, 1.0):
        assert np.abs(O.ac_step(np.full((4, 4, 4), w), 0.1, 1.0, 1.0, nsteps=5) - w).max() < 1e-15


@pytest.mark.parametrize("cbar,A,m", [(0.0, 0.4, (1, 0, 0)), (0.3, 0.25, (0, 2, 1)), (-0.2, 0.5, (1, 1, 1))])
def test_single_cosine_mode_closed_form(cbar, A, m):
    # c = cbar + A cos(k.x): c^3 - c has the modes (cos^3 = (3 cos + cos 3)/4, cos^2 = (1 + cos 2)/2)
    #   DC: cbar^3 + 3 cbar A^2 / 2 - cbar,   k: 3 cbar^2 A + 3 A^3 / 4 - A,
    #   2k: 3 cbar A^2 / 2,                    3k: A^3 / 4
    # and one step scales each by (amp - dt L g_m) / (1 + dt L kappa |m k|^2)
    n = (16, 12, 20)
    dt, L, kappa, h = 0.05, 0.9, 1.4, 0.8
    x = [np.arange(nd) for nd in n]
    X, Y, Z = np.meshgrid(*x, indexing="ij")
    phase = 2 * np.pi * (m[0] * X / n[0] + m[1] * Y / n[1] + m[2] * Z / n[2])
    c = cbar + A * np.cos(phase)
    k2 = sum((2 * np.pi * m[d] / (n[d] * h)) ** 2 for d in range(3))
    g = {0: cbar ** 3 + 1.5 * cbar * A * A - cbar, 1: 3 * cbar * cbar * A + 0.75 * A ** 3 - A,
         2: 1.5 * cbar * A * A, 3: 0.25 * A ** 3}
    amp = {0: cbar, 1: A, 2: 0.0, 3: 0.0}
    ref = np.zeros(n)
    for j in range(4):
        new = (amp[j] - dt * L * g[j]) / (1.0 + dt * L * kappa * j * j * k2)
        ref += new * (np.cos(j * phase) if j else 1.0)
    got = O.ac_step(c, dt, L, kappa, h)
    assert np.abs(got - ref).max() < 1e-13


def test_increment_form_equals_update_form():
    rng = np.random.default_rng(3)
    c = rng.uniform(-0.6, 0.6, (10, 8, 12))
    a = O.ac_step(c, 0.08, 1.1, 0.9, 1.2, nsteps=4)
    b = O.ac_step_increment(c, 0.08, 1.1, 0.9, 1.2, nsteps=4)
    assert np.abs(a - b).max() < 1e-13


def test_mean_moves_by_the_mean_of_the_nonlinearity():
    rng = np.random.default_rng(4)
    c = 0.2 + rng.uniform(-0.3, 0.3, (8, 8, 8))
    dt, L = 0.1, 1.0
    got = O.ac_step(c, dt, L, 1.0)
    assert abs(got.mean() - (c.mean() - dt * L * (c ** 3 - c).mean())) < 1e-15


@pytest.mark.parametrize("cbar", [0.0, 0.3])
def test_linearised_growth_factor(cbar):
    # a mode of amplitude eps on a uniform cbar grows by the factor
    # (1 - dt L (3 cbar^2 - 1)) / (1 + dt L kappa |k|^2) up to O(eps^2)
    n = (16, 16, 16)
    dt, L, kappa = 0.1, 1.0, 1.0
    X = np.arange(n[0])[:, None, None] * np.ones(n)
    eps = 1e-6
    c = cbar + eps * np.cos(2 * np.pi * 3 * X / n[0])
    out = O.ac_step(c, dt, L, kappa)
    k2 = (2 * np.pi * 3 / n[0]) ** 2
    amp = (out - out.mean())[:, 0, 0] @ np.cos(2 * np.pi * 3 * np.arange(n[0]) / n[0]) * 2 / n[0]
    hand = {0.0: (1.0 + 0.1) / (1.0 + 0.1 * k2), 0.3: (1.0 - 0.1 * (0.27 - 1.0)) / (1.0 + 0.1 * k2)}[cbar]
    assert abs(amp / eps - hand) < 1e-5
    assert abs(O.ac_growth_factor(k2, cbar, dt, L, kappa) - hand) < 1e-15


def test_energy_decays():
    rng = np.random.default_rng(5)
    c = rng.uniform(-0.05, 0.05, (16, 16, 16))
    _, E = O.ac_step(c, 0.1, 1.0, 1.0, nsteps=40, energies=True)
    assert np.all(np.diff(E) <= 1e-12 * np.abs(E[:-1]))
    assert E[-1] < E[0]


def test_first_order_in_dt():
    rng = np.random.default_rng(6)
    c = rng.uniform(-0.4, 0.4, (8, 8, 8))
    T = 0.4
    sol = {dt: O.ac_step(c, dt, 1.0, 1.0, nsteps=int(round(T / dt))) for dt in (0.1, 0.05, 0.025, 0.003125)}
    ref = sol[0.003125]
    e = [np.linalg.norm(sol[dt] - ref) for dt in (0.1, 0.05, 0.025)]
    for a, b in zip(e, e[1:]):
        assert 0.85 < np.log2(a / b) < 1.15


def test_ac_step_modes_matches_full_step():
    """Mode-by-mode Allen-Cahn step (direct DFT sums) equals the full FFT step."""
    from paper_2507_21748_gb300 import inputs
    c = inputs.uniform_field((16, 12, 10), seed=3, offset=0.3)
    dt, L, kappa, h = 0.1, 0.8, 1.2, 0.9
    full = O.fftn(O.ac_step(c, dt, L, kappa, h, 1))
    modes = np.array([[0, 0, 0], [1, 0, 0], [5, 7, 3], [15, 11, 9], [8, 6, 5], [2, 3, 1]])
    got = O.ac_step_modes(c, modes, dt, L, kappa, h)
    for i, (a, b, d) in enumerate(modes):
        assert abs(got[i] - full[a, b, d]) < 1e-11 * np.abs(full).max()
