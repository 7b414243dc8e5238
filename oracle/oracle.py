"""FP64 CPU oracle for the semi-implicit Fourier-spectral Cahn-Hilliard step.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference`` arm) may
import this module. The CUDA library never calls it, and it shares no code,
tables or helpers with the CUDA path.

What it computes (paper: "evoxels", Appendix "Microstructure modelling"):

* Eq. (cahn-hilliard): phi_t = div(M grad mu), mu = gamma0 g(phi) - 2 gamma0 eps lap(phi).
  With constant mobility M, the double-well derivative f'(c) = c^3 - c and
  the gradient coefficient kappa (= 2 gamma0 eps), this is
  c_t = M lap(c^3 - c - kappa lap c).
* Subsection "Semi-implicit timestepping": the stiff linear part is taken
  implicitly in Fourier space with the prefactor dt / (1 - dt S), S being the
  Fourier symbol of the linear operator (here S = -M kappa |k|^4). For the
  spectrally evaluated right-hand side -M|k|^2 (g_hat + kappa |k|^2 c_hat)
  the increment form  c^{n+1} = c^n + F^-1{ dt/(1 - dt S) F{rhs} }  equals
      c_hat^{n+1} = (c_hat^n - dt M |k|^2 g_hat^n) / (1 + dt M kappa |k|^4),
  g = c^3 - c. Both forms are implemented (``ch_step`` and
  ``ch_step_increment``) and tested against each other.
* Free energy (subsection "Phase transformations", F_int) in the c in [-1, 1]
  form: E = h^3 sum_x (c^2 - 1)^2 / 4 + h^3 (kappa/2) sum_x |grad c|^2, the
  gradient term evaluated by Parseval as (1/V) sum_k |k|^2 |c_hat(k)|^2.
* Mass: h^3 sum_x c = h^3 c_hat(0).
* Discrete adjoint of the scheme (gradients of a loss of c_N with respect to
  c_0, kappa and M): the scheme is c_{n+1} = A c_n + B g(c_n) with A, B the
  real symmetric convolutions of symbols a = 1/D, b = -dt M |k|^2 / D,
  D = 1 + dt M kappa |k|^4, so  lambda_n = A lambda_{n+1} + g'(c_n) * (B lambda_{n+1}).

* Eq. (allen-cahn), the non-conserved order parameter: phi_t = -(M/eps)
  (gamma0 g(phi) - 2 gamma0 eps lap phi). Under the same readings (gamma0 = 1,
  kappa = 2 gamma0 eps, double well f'(c) = c^3 - c, kinetic coefficient L
  standing for M/eps) this is c_t = -L (c^3 - c - kappa lap c). The same
  semi-implicit recipe with S = -L kappa |k|^2 (the subsection applies it "to
  all reaction-diffusion and phase evolution problems") gives
      c_hat^{n+1} = (c_hat^n - dt L g_hat^n) / (1 + dt L kappa |k|^2),
  with no |k|^2 in front of g_hat, so the mean moves:
      mean(c^{n+1}) = mean(c^n) - dt L mean(g(c^n)).
  ``ac_step`` and ``ac_step_increment`` implement the two forms.

* The general form of subsection "Semi-implicit timestepping": the
  right-hand side is coded as a finite-difference approximation in real space
  and only the preconditioner dt / (1 - dt S0) is spectral,
      c^{n+1} = c^n + F^-1{ dt / (1 + dt M kappa |k|^4) F{rhs(c^n)} },
  here for Eq. (cahn-hilliard) with the variable mobility of that equation,
  M(phi) = D0 phi (1 - phi), read in the c form as M(c) = M max(1 - c^2, 0)
  (D0 = 4 M under phi = (1 + c)/2, clipped at 0 so the operator stays
  dissipative where c overshoots the wells). rhs = div(M(c) grad mu),
  mu = c^3 - c - kappa lap_h c, with second-order central differences in
  conservative form: lap_h the 7-point Laplacian and
      div(M grad mu)_i = sum_d [M_{i+e_d/2} (mu_{i+e_d} - mu_i)
                                - M_{i-e_d/2} (mu_i - mu_{i-e_d})] / h^2,
      M_{i+e_d/2} = (M_i + M_{i+e_d}) / 2.
  ``vm_rhs``, ``vm_step`` and ``vm_energy`` (FD gradient energy) implement it.

Transforms: forward F(u)(k) = sum_x u(x) exp(-i k.x), inverse with
exp(+i k.x) and 1/V, computed by the oracle's own textbook mixed-radix FFT in
``evx_oracle.c`` (full complex 3D, no real-to-complex shortcut).
Wave numbers: k_d(m) = 2 pi m~ / (N_d h), m~ = m for m <= N_d/2 else m - N_d
(the spectral wave number; only even powers of k occur so the sign of the
Nyquist mode does not matter).
"""
import ctypes
import os

import numpy as np

from .build import build_oracle

_lib = None


def _L():
    global _lib
    if _lib is None:
        path = build_oracle()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.orc_fft1d.argtypes = [dp, ctypes.c_int, ctypes.c_int]
        lib.orc_fft3d.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.orc_dft_modes.argtypes = [fp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ip, ctypes.c_int, dp, dp]
        lib.orc_vm_rhs_modes.argtypes = [fp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_int, ip, dp, dp]
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_L().orc_num_threads())


# ---------------------------------------------------------------- transforms
def fft1d(u, sign=-1):
    """Unnormalised 1D DFT, sign -1 forward, +1 inverse (no 1/N)."""
    a = np.ascontiguousarray(np.asarray(u, dtype=np.complex128)).copy()
    _L().orc_fft1d(a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a.size, int(sign))
    return a


def fftn(u, sign=-1):
    """Unnormalised 3D DFT of a C-order (nx, ny, nz) array; sign -1 forward."""
    a = np.ascontiguousarray(np.asarray(u, dtype=np.complex128)).copy()
    nx, ny, nz = a.shape
    _L().orc_fft3d(a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nx, ny, nz, int(sign))
    return a


def ifftn(uh):
    """Inverse 3D DFT including the 1/V normalisation."""
    a = fftn(uh, +1)
    a /= a.size
    return a


# ------------------------------------------------------------ wave numbers
def wavenumbers(n, h=1.0):
    """k(m) = 2 pi m~ / (n h), m~ the signed index (m - n for m > n/2)."""
    m = np.arange(n, dtype=np.float64)
    m = np.where(m <= n // 2, m, m - n)
    return 2.0 * np.pi * m / (n * h)


def k2_grid(shape, h=1.0):
    nx, ny, nz = shape
    kx, ky, kz = wavenumbers(nx, h), wavenumbers(ny, h), wavenumbers(nz, h)
    return kx[:, None, None] ** 2 + ky[None, :, None] ** 2 + kz[None, None, :] ** 2


def symbols(shape, dt, M, kappa, h=1.0):
    """a = 1/D and b = -dt M |k|^2 / D with D = 1 + dt M kappa |k|^4."""
    k2 = k2_grid(shape, h)
    D = 1.0 + dt * M * kappa * k2 * k2
    return 1.0 / D, -dt * M * k2 / D, k2, D


# ------------------------------------------------------------------ scheme
def fprime(c):
    """Pointwise chemical-potential term f'(c) = c^3 - c (double well)."""
    return c * c * c - c


def ch_step(c, dt, M, kappa, h=1.0, nsteps=1, energies=False, check_imag=True):
    """Advance c by nsteps semi-implicit spectral steps (FP64).

    Per step:  c_hat = F c;  g = c^3 - c;  g_hat = F g;
               c_hat' = (c_hat - dt M |k|^2 g_hat) / (1 + dt M kappa |k|^4);
               c' = Re F^-1 c_hat'.
    Returns c (float64) and, if ``energies``, the energy after every step
    (index 0 = initial energy).
    """
    c = np.asarray(c, dtype=np.float64).copy()
    a, b, k2, _ = symbols(c.shape, dt, M, kappa, h)
    E = [energy(c, kappa, h)] if energies else None
    for _ in range(nsteps):
        c_hat = fftn(c)
        g_hat = fftn(fprime(c))
        c_new = ifftn((c_hat - dt * M * k2 * g_hat) / (1.0 + dt * M * kappa * k2 * k2))
        if check_imag:
            scale = max(np.abs(c).max(), 1e-300)
            assert np.abs(c_new.imag).max() < 1e-12 * scale + 1e-300, "non-real inverse transform"
        c = c_new.real.copy()
        if energies:
            E.append(energy(c, kappa, h))
    return (c, np.array(E)) if energies else c


def ch_step_increment(c, dt, M, kappa, h=1.0, nsteps=1):
    """The appendix's increment form: c' = c + F^-1{ dt / (1 - dt S) F{rhs} },
    S = -M kappa |k|^4 and rhs evaluated spectrally as
    F{rhs} = -M |k|^2 (g_hat + kappa |k|^2 c_hat)."""
    c = np.asarray(c, dtype=np.float64).copy()
    k2 = k2_grid(c.shape, h)
    S = -M * kappa * k2 * k2
    for _ in range(nsteps):
        c_hat = fftn(c)
        g_hat = fftn(fprime(c))
        rhs_hat = -M * k2 * (g_hat + kappa * k2 * c_hat)
        c = c + ifftn(dt / (1.0 - dt * S) * rhs_hat).real
    return c


def ch_block_step(c, dt, M, kappa, h=1.0, nsteps=10):
    """One block of nsteps steps of the scheme with its stiff linear part exact
    and its nonlinear remainder frozen at the block's start (the learned
    surrogate's base propagator; a construct of this build, not the paper's).

    Write the scheme's update (subsection "Semi-implicit timestepping",
    S = -M kappa |k|^4) as c_hat' = (c_hat - dt M |k|^2 g_hat) / D and split
    g(c) = g(cbar) + g'(cbar) d + N(d), d = c - cbar, N = d^2 (3 cbar + d). The
    part linear in d is one multiplication per mode,
        c_hat' = L c_hat + B N_hat,  L = (1 - dt M |k|^2 g'(cbar)) / D,  B = -dt M |k|^2 / D,
    (k != 0; the mean cbar is conserved). Holding N_hat fixed over nsteps steps:
        d_hat_n = L^n d_hat_0 + B (sum_{j<n} L^j) N_hat_0.
    nsteps = 1 is exactly one step of the scheme.
    """
    c = np.asarray(c, dtype=np.float64)
    cb = float(c.mean())
    a, b, k2, D = symbols(c.shape, dt, M, kappa, h)
    Lk = (1.0 - dt * M * k2 * (3.0 * cb * cb - 1.0)) / D
    d = c - cb
    P = np.ones_like(Lk)
    Ssum = np.zeros_like(Lk)
    for _ in range(nsteps):
        Ssum += P
        P = P * Lk
    dh = P * fftn(d) + b * Ssum * fftn(d * d * (3.0 * cb + d))
    dh[0, 0, 0] = 0.0
    return cb + ifftn(dh).real


def ac_step(c, dt, L, kappa, h=1.0, nsteps=1, energies=False, check_imag=True):
    """Advance c by nsteps semi-implicit spectral Allen-Cahn steps (FP64).

    Per step:  c_hat = F c;  g_hat = F(c^3 - c);
               c_hat' = (c_hat - dt L g_hat) / (1 + dt L kappa |k|^2);
               c' = Re F^-1 c_hat'.
    Returns c (float64) and, if ``energies``, the energy after every step.
    """
    c = np.asarray(c, dtype=np.float64).copy()
    k2 = k2_grid(c.shape, h)
    E = [energy(c, kappa, h)] if energies else None
    for _ in range(nsteps):
        c_hat = fftn(c)
        g_hat = fftn(fprime(c))
        c_new = ifftn((c_hat - dt * L * g_hat) / (1.0 + dt * L * kappa * k2))
        if check_imag:
            scale = max(np.abs(c).max(), 1e-300)
            assert np.abs(c_new.imag).max() < 1e-12 * scale + 1e-300, "non-real inverse transform"
        c = c_new.real.copy()
        if energies:
            E.append(energy(c, kappa, h))
    return (c, np.array(E)) if energies else c


def ac_step_increment(c, dt, L, kappa, h=1.0, nsteps=1):
    """Increment form c' = c + F^-1{ dt / (1 - dt S) F{rhs} } for Allen-Cahn,
    S = -L kappa |k|^2 and F{rhs} = -L (g_hat + kappa |k|^2 c_hat)."""
    c = np.asarray(c, dtype=np.float64).copy()
    k2 = k2_grid(c.shape, h)
    S = -L * kappa * k2
    for _ in range(nsteps):
        c_hat = fftn(c)
        g_hat = fftn(fprime(c))
        rhs_hat = -L * (g_hat + kappa * k2 * c_hat)
        c = c + ifftn(dt / (1.0 - dt * S) * rhs_hat).real
    return c


def ac_growth_factor(k2, cbar, dt, L, kappa):
    """Allen-Cahn amplification per step of a small mode on a uniform cbar."""
    return (1.0 - dt * L * (3.0 * cbar * cbar - 1.0)) / (1.0 + dt * L * kappa * k2)


def vm_mobility(c, M):
    """M(c) = M max(1 - c^2, 0)."""
    return M * np.maximum(1.0 - c * c, 0.0)


def lap_h(u, h=1.0):
    """7-point periodic Laplacian (second-order central differences)."""
    out = -6.0 * u
    for ax in range(3):
        out = out + np.roll(u, 1, axis=ax) + np.roll(u, -1, axis=ax)
    return out / (h * h)


def vm_rhs(c, M, kappa, h=1.0, mobility=None):
    """div(M(c) grad mu), mu = c^3 - c - kappa lap_h c, conservative central
    differences with face mobilities (M_i + M_{i+e_d}) / 2. ``mobility`` (a
    function of c) replaces M(c) = M max(1 - c^2, 0) when given."""
    c = np.asarray(c, dtype=np.float64)
    mu = fprime(c) - kappa * lap_h(c, h)
    Mc = vm_mobility(c, M) if mobility is None else mobility(c)
    out = np.zeros_like(c)
    for ax in range(3):
        mu_p, M_p = np.roll(mu, -1, axis=ax), np.roll(Mc, -1, axis=ax)
        flux = 0.5 * (Mc + M_p) * (mu_p - mu)  # on the face i + e_d/2
        out = out + flux - np.roll(flux, 1, axis=ax)
    return out / (h * h)


def vm_step(c, dt, M, kappa, h=1.0, nsteps=1, mobility=None, M0=None, energies=False):
    """nsteps of c' = c + F^-1{ dt / (1 + dt M0 kappa |k|^4) F{rhs(c)} }, M0 = M by default."""
    c = np.asarray(c, dtype=np.float64).copy()
    k2 = k2_grid(c.shape, h)
    pref = dt / (1.0 + dt * (M if M0 is None else M0) * kappa * k2 * k2)
    E = [vm_energy(c, kappa, h)] if energies else None
    for _ in range(nsteps):
        c = c + ifftn(pref * fftn(vm_rhs(c, M, kappa, h, mobility))).real
        if energies:
            E.append(vm_energy(c, kappa, h))
    return (c, np.array(E)) if energies else c


def vm_energy(c, kappa, h=1.0):
    """h^3 sum (c^2-1)^2/4 + h^3 (kappa/2) sum_d sum ((c_{i+e_d} - c_i)/h)^2."""
    c = np.asarray(c, dtype=np.float64)
    bulk = np.sum((c * c - 1.0) ** 2) / 4.0
    grad = sum(np.sum((np.roll(c, -1, axis=ax) - c) ** 2) for ax in range(3)) / (h * h)
    return h ** 3 * (bulk + 0.5 * kappa * grad)


def energy(c, kappa, h=1.0):
    """Ginzburg-Landau energy h^3 sum (c^2-1)^2/4 + h^3 (kappa/2)(1/V) sum_k |k|^2 |c_hat|^2."""
    c = np.asarray(c, dtype=np.float64)
    V = c.size
    bulk = np.sum((c * c - 1.0) ** 2) / 4.0
    c_hat = fftn(c)
    grad = np.sum(k2_grid(c.shape, h) * np.abs(c_hat) ** 2) / V
    return h ** 3 * (bulk + 0.5 * kappa * grad)


def mass(c, h=1.0):
    return h ** 3 * float(np.sum(np.asarray(c, dtype=np.float64)))


def growth_factor(k2, cbar, dt, M, kappa):
    """Amplification per step of a small mode on a uniform background cbar
    (the scheme linearised about cbar: g'(cbar) = 3 cbar^2 - 1)."""
    return (1.0 - dt * M * k2 * (3.0 * cbar * cbar - 1.0)) / (1.0 + dt * M * kappa * k2 * k2)


# ------------------------------------------------ single modes of big grids
def dft_modes(c32, modes, which="c"):
    """Direct sums sum_x f(c(x)) exp(-i k.x) at integer wave vectors.

    c32: float32 (nx, ny, nz); modes: (n, 3) ints; which 'c' (f = c) or
    'g' (f = c^3 - c). FP64 accumulation, O(V) per call."""
    c32 = np.ascontiguousarray(c32, dtype=np.float32)
    md = np.ascontiguousarray(np.asarray(modes, dtype=np.int32).reshape(-1, 3))
    n = md.shape[0]
    re = np.zeros(n)
    im = np.zeros(n)
    nx, ny, nz = c32.shape
    _L().orc_dft_modes(c32.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), nx, ny, nz, n,
                       md.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), 1 if which == "g" else 0,
                       re.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       im.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return re + 1j * im


def step_modes(c32, modes, dt, M, kappa, h=1.0):
    """c_hat^{n+1}(k) for selected k after one step from c32, each mode
    computed on its own from the definition (direct DFT sums of c and c^3-c)."""
    md = np.asarray(modes, dtype=np.int64).reshape(-1, 3)
    shape = c32.shape
    k2 = np.zeros(md.shape[0])
    for d in range(3):
        k2 += wavenumbers(shape[d], h)[md[:, d] % shape[d]] ** 2
    ch = dft_modes(c32, md, "c")
    gh = dft_modes(c32, md, "g")
    return (ch - dt * M * k2 * gh) / (1.0 + dt * M * kappa * k2 * k2)


def _mode_k2(shape, md, h):
    k2 = np.zeros(md.shape[0])
    for d in range(3):
        k2 += wavenumbers(shape[d], h)[md[:, d] % shape[d]] ** 2
    return k2


def ac_step_modes(c32, modes, dt, L, kappa, h=1.0):
    """Allen-Cahn c_hat^{n+1}(k) = (c_hat - dt L g_hat) / (1 + dt L kappa |k|^2) at
    selected k after one step from c32, each mode from direct DFT sums."""
    md = np.asarray(modes, dtype=np.int64).reshape(-1, 3)
    k2 = _mode_k2(c32.shape, md, h)
    ch = dft_modes(c32, md, "c")
    gh = dft_modes(c32, md, "g")
    return (ch - dt * L * gh) / (1.0 + dt * L * kappa * k2)


def vm_rhs_modes(c32, modes, M, kappa, h=1.0):
    """sum_x rhs(x) exp(-i k.x) of the variable-mobility FD right-hand side
    (``vm_rhs``), formed plane by plane in C (no full-size FP64 arrays)."""
    c32 = np.ascontiguousarray(c32, dtype=np.float32)
    md = np.ascontiguousarray(np.asarray(modes, dtype=np.int32).reshape(-1, 3))
    n = md.shape[0]
    re = np.zeros(n)
    im = np.zeros(n)
    nx, ny, nz = c32.shape
    _L().orc_vm_rhs_modes(c32.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), nx, ny, nz, float(M), float(kappa),
                          float(h), n, md.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                          re.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          im.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return re + 1j * im


def vm_step_modes(c32, modes, dt, M, kappa, h=1.0):
    """Variable-mobility c_hat^{n+1}(k) = c_hat + dt / (1 + dt M kappa |k|^4) rhs_hat
    at selected k after one step from c32."""
    md = np.asarray(modes, dtype=np.int64).reshape(-1, 3)
    k2 = _mode_k2(c32.shape, md, h)
    return dft_modes(c32, md, "c") + dt / (1.0 + dt * M * kappa * k2 * k2) * vm_rhs_modes(c32, md, M, kappa, h)


# ---------------------------------------------------------------- adjoint
def ch_forward_states(c0, dt, M, kappa, h, nsteps):
    """States c_0 .. c_N of the scheme (list of float64 arrays)."""
    cs = [np.asarray(c0, dtype=np.float64).copy()]
    for _ in range(nsteps):
        cs.append(ch_step(cs[-1], dt, M, kappa, h, 1, check_imag=False))
    return cs


def ch_tangent(c0, dc0, dt, M, kappa, h, nsteps, dkappa=0.0, dM=0.0):
    """Tangent-linear model: derivative of c_N along (dc0, dkappa, dM)."""
    c = np.asarray(c0, dtype=np.float64).copy()
    dc = np.asarray(dc0, dtype=np.float64).copy()
    k2 = k2_grid(c.shape, h)
    for _ in range(nsteps):
        D = 1.0 + dt * M * kappa * k2 * k2
        a = 1.0 / D
        b = -dt * M * k2 / D
        # partial derivatives of the symbols
        da_dk = -dt * M * k2 * k2 / D ** 2
        db_dk = dt * dt * M * M * k2 ** 3 / D ** 2
        da_dM = -dt * kappa * k2 * k2 / D ** 2
        db_dM = -dt * k2 / D ** 2
        c_hat = fftn(c)
        g_hat = fftn(fprime(c))
        dc_hat = fftn(dc)
        dg_hat = fftn((3.0 * c * c - 1.0) * dc)
        new_dc = (a * dc_hat + b * dg_hat
                  + dkappa * (da_dk * c_hat + db_dk * g_hat)
                  + dM * (da_dM * c_hat + db_dM * g_hat))
        c = ifftn(a * c_hat + b * g_hat).real
        dc = ifftn(new_dc).real
    return dc


def ch_adjoint(c0, dLdcN, dt, M, kappa, h, nsteps):
    """Discrete adjoint of ``ch_step`` (all states kept in memory).

    lambda_N = dL/dc_N; for n = N-1 .. 0 with lambda_hat = F lambda_{n+1}:
      dL/dkappa += (1/V) sum_k Re[conj(lambda_hat) (da/dkappa c_hat_n + db/dkappa g_hat_n)]
      dL/dM     += (1/V) sum_k Re[conj(lambda_hat) (da/dM c_hat_n + db/dM g_hat_n)]
      lambda_n = F^-1(a lambda_hat) + (3 c_n^2 - 1) F^-1(b lambda_hat)
    with da/dkappa = -dt M k^4/D^2, db/dkappa = dt^2 M^2 k^6/D^2,
    da/dM = -dt kappa k^4/D^2, db/dM = -dt k^2/D^2.
    Returns (dL/dc_0, dL/dkappa, dL/dM).
    """
    cs = ch_forward_states(c0, dt, M, kappa, h, nsteps)
    k2 = k2_grid(cs[0].shape, h)
    V = cs[0].size
    D = 1.0 + dt * M * kappa * k2 * k2
    a = 1.0 / D
    b = -dt * M * k2 / D
    da_dk = -dt * M * k2 * k2 / D ** 2
    db_dk = dt * dt * M * M * k2 ** 3 / D ** 2
    da_dM = -dt * kappa * k2 * k2 / D ** 2
    db_dM = -dt * k2 / D ** 2
    lam = np.asarray(dLdcN, dtype=np.float64).copy()
    gk = 0.0
    gM = 0.0
    for n in range(nsteps - 1, -1, -1):
        c = cs[n]
        lam_hat = fftn(lam)
        c_hat = fftn(c)
        g_hat = fftn(fprime(c))
        cl = np.conj(lam_hat)
        gk += float(np.sum((cl * (da_dk * c_hat + db_dk * g_hat)).real)) / V
        gM += float(np.sum((cl * (da_dM * c_hat + db_dM * g_hat)).real)) / V
        lam = ifftn(a * lam_hat).real + (3.0 * c * c - 1.0) * ifftn(b * lam_hat).real
    return lam, gk, gM
