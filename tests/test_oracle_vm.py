"""Pins for the oracle's variable-mobility Cahn-Hilliard step (test
infrastructure): the general form of "Semi-implicit timestepping" with a
finite-difference right-hand side div(M(c) grad mu) and the spectral
preconditioner dt / (1 + dt M kappa |k|^4).

The FD operator is pinned by a brute-force loop written from the stencil's
definition, its conservation, and a constant-mobility closed form built from
the FD symbols of a cosine mode; the step by first order in dt and energy
decay; the FD energy by the closed form of a cosine mode."""
import numpy as np
import pytest

from oracle import oracle as O


def brute_rhs(c, M, kappa, h):
    X, Y, Z = c.shape
    mob = lambda v: M * max(1.0 - v * v, 0.0)

    def at(i, j, k):
        return c[i % X, j % Y, k % Z]

    def mu(i, j, k):
        v = at(i, j, k)
        lap = (at(i + 1, j, k) + at(i - 1, j, k) + at(i, j + 1, k) + at(i, j - 1, k) + at(i, j, k + 1)
               + at(i, j, k - 1) - 6.0 * v) / (h * h)
        return v ** 3 - v - kappa * lap

    out = np.zeros(c.shape)
    for i in range(X):
        for j in range(Y):
            for k in range(Z):
                acc = 0.0
                for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
                    ip = (i + d[0], j + d[1], k + d[2])
                    im = (i - d[0], j - d[1], k - d[2])
                    Mp = 0.5 * (mob(at(i, j, k)) + mob(at(*ip)))
                    Mm = 0.5 * (mob(at(i, j, k)) + mob(at(*im)))
                    acc += Mp * (mu(*ip) - mu(i, j, k)) - Mm * (mu(i, j, k) - mu(*im))
                out[i, j, k] = acc / (h * h)
    return out


def test_rhs_against_brute_force_loop():
    rng = np.random.default_rng(0)
    c = rng.uniform(-1.1, 1.1, (5, 4, 6))  # includes |c| > 1, where the mobility clips at 0
    got = O.vm_rhs(c, 0.8, 1.3, 0.9)
    ref = brute_rhs(c, 0.8, 1.3, 0.9)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_rhs_conserves_mass_and_uniform_fields_are_fixed():
    rng = np.random.default_rng(1)
    c = rng.uniform(-0.9, 0.9, (8, 6, 10))
    r = O.vm_rhs(c, 1.0, 1.0, 1.0)
    assert abs(r.sum()) < 1e-12 * np.abs(r).sum()
    assert np.abs(O.vm_rhs(np.full((4, 4, 4), 0.3), 1.0, 1.0)).max() == 0.0


def test_constant_mobility_cosine_mode_closed_form():
    # with M(c) = M0 constant, rhs = M0 lap_h (c^3 - c) - M0 kappa lap_h^2 c and a mode
    # cos(j k.x) is an eigenfunction of lap_h with eigenvalue -kt_j^2,
    # kt^2 = sum_d (2 - 2 cos(j k_d h)) / h^2; c^3 - c of c = cbar + A cos has the modes
    # DC: cbar^3 + 3 cbar A^2/2 - cbar, 1: 3 cbar^2 A + 3A^3/4 - A, 2: 3 cbar A^2/2, 3: A^3/4.
    # One step: amp_j' = amp_j + dt (-M0 kt_j^2 (g_j + kappa kt_j^2 amp_j)) / (1 + dt M0 kappa k_j^4)
    n = (16, 12, 20)
    m = (1, 2, 1)
    cbar, A = 0.2, 0.3
    dt, M0, kappa, h = 0.05, 0.9, 1.2, 0.8
    X, Y, Z = np.meshgrid(*[np.arange(nd) for nd in n], indexing="ij")
    phase = 2 * np.pi * (m[0] * X / n[0] + m[1] * Y / n[1] + m[2] * Z / n[2])
    c = cbar + A * np.cos(phase)
    g = {0: cbar ** 3 + 1.5 * cbar * A * A - cbar, 1: 3 * cbar * cbar * A + 0.75 * A ** 3 - A,
         2: 1.5 * cbar * A * A, 3: 0.25 * A ** 3}
    amp = {0: cbar, 1: A, 2: 0.0, 3: 0.0}
    ref = np.zeros(n)
    for j in range(4):
        kd = [2 * np.pi * j * m[d] / (n[d] * h) for d in range(3)]
        kt2 = sum((2 - 2 * np.cos(q * h)) / h ** 2 for q in kd)
        ks2 = sum(q * q for q in kd)
        new = amp[j] + dt * (-M0 * kt2 * (g[j] + kappa * kt2 * amp[j])) / (1 + dt * M0 * kappa * ks2 * ks2)
        ref += new * (np.cos(j * phase) if j else 1.0)
    got = O.vm_step(c, dt, M0, kappa, h, mobility=lambda v: M0 + 0.0 * v)
    assert np.abs(got - ref).max() < 1e-13


def test_first_order_in_dt():
    # h = 4 keeps dt M kappa |k|^4 small for every mode, so the steps sit in the
    # asymptotic regime; successive differences halve with dt (first order)
    rng = np.random.default_rng(2)
    c = 0.1 + rng.uniform(-0.3, 0.3, (8, 8, 8))
    T, h = 0.8, 4.0
    dts = (0.1, 0.05, 0.025, 0.0125, 0.00625)
    sol = {dt: O.vm_step(c, dt, 1.0, 1.0, h, nsteps=int(round(T / dt))) for dt in dts}
    e = [np.linalg.norm(sol[a] - sol[b]) for a, b in zip(dts, dts[1:])]
    orders = [np.log2(a / b) for a, b in zip(e, e[1:])]
    assert all(0.85 < q < 1.15 for q in orders[1:])
    assert orders[-1] > orders[0]  # approaching 1 from below


def test_mass_conserved_and_energy_decays():
    rng = np.random.default_rng(3)
    c = 0.1 + rng.uniform(-0.05, 0.05, (16, 16, 16))
    out, E = O.vm_step(c, 0.1, 1.0, 1.0, nsteps=30, energies=True)
    assert abs(out.mean() - c.mean()) < 1e-14
    assert np.all(np.diff(E) <= 1e-12 * np.abs(E[:-1]))
    assert E[-1] < E[0]


@pytest.mark.parametrize("h", [1.0, 0.8])
@pytest.mark.parametrize("m", [(2, 0, 0), (1, 2, 3)])
def test_vm_energy_closed_form_cosine_mode(m, h):
    """FD energy of c = A cos(k.x), k_d = 2 pi m_d / (n_d h), on an n-grid of edge h:
      bulk     h^3 sum (c^2 - 1)^2 / 4 = h^3 V (3A^4/8 - A^2 + 1) / 4
               (means of cos^2 and cos^4 over whole periods: 1/2 and 3/8),
      gradient h^3 (kappa/2) sum_d sum_x ((c(x + h e_d) - c(x)) / h)^2
               = h^3 (kappa/2) V A^2 sum_d (1 - cos(k_d h)) / h^2,
    since cos(t + q) - cos t = -2 sin(q/2) sin(t + q/2) and the mean of sin^2 is 1/2.
    A gradient weight of kappa instead of kappa/2, a missing h^3 or 1/h^2, or a
    central instead of a forward difference each change the value."""
    n, A, kappa = (16, 12, 20), 0.35, 1.3
    X, Y, Z = np.meshgrid(*[np.arange(nd) for nd in n], indexing="ij")
    c = A * np.cos(2 * np.pi * (m[0] * X / n[0] + m[1] * Y / n[1] + m[2] * Z / n[2]))
    V = n[0] * n[1] * n[2]
    kh = [2 * np.pi * m[d] / n[d] for d in range(3)]  # k_d h
    bulk = h ** 3 * V * (3 * A ** 4 / 8 - A ** 2 + 1) / 4
    grad = h ** 3 * 0.5 * kappa * V * A ** 2 * sum((1 - np.cos(q)) / h ** 2 for q in kh)
    got = O.vm_energy(c, kappa, h)
    assert abs(got - (bulk + grad)) < 1e-11 * (bulk + grad)


def test_vm_rhs_modes_and_step_modes_match_full_arrays():
    """The plane-by-plane C sums of the FD right-hand side equal the FFT of the
    numpy right-hand side (itself pinned by the brute-force loop), and the
    mode-by-mode step equals the full step, at every sampled mode."""
    from paper_2507_21748_gb300 import inputs
    c = inputs.uniform_field((10, 12, 14), seed=4, offset=0.2, lo=-0.9, hi=0.9)  # |c| > 1 clips M
    M, kappa, h, dt = 0.8, 1.3, 0.9, 0.05
    modes = np.array([[0, 0, 0], [1, 0, 0], [0, 3, 7], [9, 11, 13], [5, 6, 7], [2, 1, 4]])
    full_rhs = O.fftn(O.vm_rhs(c, M, kappa, h))
    got = O.vm_rhs_modes(c, modes, M, kappa, h)
    full_step = O.fftn(O.vm_step(c, dt, M, kappa, h))
    got_step = O.vm_step_modes(c, modes, dt, M, kappa, h)
    for i, (a, b, d) in enumerate(modes):
        assert abs(got[i] - full_rhs[a, b, d]) < 1e-11 * np.abs(full_rhs).max()
        assert abs(got_step[i] - full_step[a, b, d]) < 1e-11 * np.abs(full_step).max()
