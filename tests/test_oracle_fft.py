"""Pins for the oracle's textbook FFT (test infrastructure).

The semi-implicit step (Appendix "Semi-implicit timestepping") needs the
forward transform F{u}(k) = sum_x u(x) exp(-i k.x) and its inverse. The
oracle's FFT is checked against a brute-force O(N^2) DFT written from the
definition, against numpy.fft (a library routine), and for round trip.
"""
import numpy as np
import pytest

from oracle import oracle as O


def brute_dft_1d(u, sign=-1):
    n = len(u)
    j = np.arange(n)
    W = np.exp(sign * 2j * np.pi * np.outer(j, j) / n)
    return W @ u


@pytest.mark.parametrize("n", [2, 3, 5, 8, 12, 25, 80, 400, 7, 49])
def test_fft1d_vs_bruteforce(n):
    rng = np.random.default_rng(n)
    u = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for sign in (-1, 1):
        ref = brute_dft_1d(u, sign)
        got = O.fft1d(u, sign)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_fft3d_vs_bruteforce_8cubed():
    rng = np.random.default_rng(8)
    u = rng.standard_normal((8, 8, 8))
    # brute force: the full 512x512 DFT matrix of the flattened index
    idx = np.indices((8, 8, 8)).reshape(3, -1).T
    phase = (idx @ idx.T) / 8.0  # (x . k) / N with N = 8 on every axis
    W = np.exp(-2j * np.pi * phase)
    ref = (W @ u.reshape(-1)).reshape(8, 8, 8)
    got = O.fftn(u)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("shape", [(8, 12, 10), (16, 16, 16), (6, 20, 25)])
def test_fft3d_vs_numpy(shape):
    rng = np.random.default_rng(1)
    u = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    assert np.abs(O.fftn(u) - np.fft.fftn(u)).max() <= 1e-12 * np.abs(u).sum() ** 0.5 * 10
    assert np.allclose(O.fftn(u, +1), np.fft.ifftn(u) * u.size, rtol=0, atol=1e-11)


@pytest.mark.parametrize("shape", [(8, 8, 8), (10, 12, 16)])
def test_roundtrip(shape):
    rng = np.random.default_rng(2)
    u = rng.standard_normal(shape)
    back = O.ifftn(O.fftn(u))
    assert np.abs(back - u).max() <= 1e-14 * max(1.0, np.abs(u).max()) * 10
    assert np.abs(back.imag).max() < 1e-14


def test_dft_modes_vs_fft():
    rng = np.random.default_rng(3)
    c = (rng.random((12, 10, 8)) * 0.2 - 0.1).astype(np.float32)
    full_c = O.fftn(c.astype(np.float64))
    full_g = O.fftn(O.fprime(c.astype(np.float64)))
    modes = np.array([[0, 0, 0], [1, 2, 3], [11, 9, 7], [6, 5, 4], [3, 0, 1]])
    got_c = O.dft_modes(c, modes, "c")
    got_g = O.dft_modes(c, modes, "g")
    for i, (a, b, d) in enumerate(modes):
        assert abs(got_c[i] - full_c[a, b, d]) < 1e-12
        assert abs(got_g[i] - full_g[a, b, d]) < 1e-12
