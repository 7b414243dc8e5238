"""The FMA forms of the register DFTs in csrc/evx_fft.cuh and of the real-transform
pre/post-processing in csrc/evx_fast_dev.cuh, restated operation by operation in
FP64 and checked against numpy's FFT (host logic, no GPU). They are the forms the
issue-bound x and z passes run; a sign, twiddle or index slip in them fails here.
"""
import numpy as np
import pytest

C1, S1, R2 = np.cos(np.pi / 8), np.sin(np.pi / 8), np.cos(np.pi / 4)
TAB16 = {1: (C1, S1), 2: (R2, R2), 3: (S1, C1), 5: (-S1, C1), 6: (-R2, R2), 7: (-C1, S1)}


def mul_i(d, a):  # multiply by -i (d = -1) or +i (d = +1)
    return complex(a.imag, -a.real) if d < 0 else complex(-a.imag, a.real)


def w16(d, m, a):  # a exp(d i pi m / 8), m < 8, as the general complex product
    if m == 0:
        return a
    if m == 4:
        return mul_i(d, a)
    c, s = TAB16[m]
    ds = -s if d < 0 else s
    return complex(a.real * c - a.imag * ds, a.real * ds + a.imag * c)


def tw16_fma(d, m, a, b):  # b + w^m a, two FMAs per component; w^(m+8) = -w^m
    mm, sg = m & 7, (-1.0 if m & 8 else 1.0)
    if mm == 0:
        return b + a if sg > 0 else b - a
    if mm == 4:
        return b + mul_i(d, a) if sg > 0 else b - mul_i(d, a)
    c0, s0 = TAB16[mm]
    c, ds = sg * c0, (-sg * s0 if d < 0 else sg * s0)
    return complex(c * a.real - ds * a.imag + b.real, c * a.imag + ds * a.real + b.imag)


def dft4(d, a0, a1, a2, a3):
    t0, t1, t2, t3 = a0 + a2, a0 - a2, a1 + a3, mul_i(d, a1 - a3)
    return t0 + t2, t1 + t3, t0 - t2, t1 - t3


def dft4_tw(d, m1, m2, m3, a0, a1, a2, a3):
    if (m2 & 3) == 0:
        r = mul_i(d, a2) if m2 & 4 else a2
        b2 = -r if m2 & 8 else r
        t0, t1 = a0 + b2, a0 - b2
    else:
        t0 = tw16_fma(d, m2, a2, a0)
        t1 = 2 * a0 - t0
    u1 = w16(d, m1, a1)
    t2 = tw16_fma(d, m3, a3, u1)
    t3 = mul_i(d, 2 * u1 - t2)
    return t0 + t2, t1 + t3, t0 - t2, t1 - t3


def dft16(d, x):
    v = list(x)
    for n2 in range(4):
        v[n2], v[4 + n2], v[8 + n2], v[12 + n2] = dft4(d, v[n2], v[4 + n2], v[8 + n2], v[12 + n2])
    v[0:4] = dft4(d, *v[0:4])
    v[4:8] = dft4_tw(d, 1, 2, 3, *v[4:8])
    v[8:12] = dft4_tw(d, 2, 4, 6, *v[8:12])
    v[12:16] = dft4_tw(d, 3, 6, 9, *v[12:16])
    return np.array([v[4 * (k % 4) + k // 4] for k in range(16)])  # slot 4 k1 + k2 holds X[k1 + 4 k2]


def dft32(d, x):
    e, o = dft16(d, x[0::2]), dft16(d, x[1::2])
    out = np.zeros(32, dtype=complex)
    for k in range(16):
        if k in (0, 8):
            t = o[k] if k == 0 else mul_i(d, o[k])
            out[k], out[k + 16] = e[k] + t, e[k] - t
            continue
        c, sn = np.cos(np.pi * k / 16), np.sin(np.pi * k / 16)
        ds = -sn if d < 0 else sn
        s = complex(c * o[k].real - ds * o[k].imag + e[k].real, c * o[k].imag + ds * o[k].real + e[k].imag)
        out[k], out[k + 16] = s, 2 * e[k] - s
    return out


@pytest.mark.parametrize("d", [-1, 1])
def test_dft16_and_dft32_fma_forms(d):
    rng = np.random.default_rng(7 + d)
    for n, f in ((16, dft16), (32, dft32)):
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        ref = np.fft.fft(x) if d < 0 else np.fft.ifft(x) * n
        assert np.abs(f(d, x) - ref).max() < 1e-12 * n


def c2r_pre(xk, xm, w):
    px, py, qx, qy = xk.real + xm.real, xk.imag - xm.imag, xk.real - xm.real, xk.imag + xm.imag
    return complex(-w.real * qy + w.imag * qx + px, w.real * qx + w.imag * qy + py)


def r2c_post(zk, zm, w):
    px, py, qx, qy = zk.real + zm.real, zk.imag - zm.imag, zk.real - zm.real, zk.imag + zm.imag
    return complex(0.5 * (w.real * qy + w.imag * qx + px), 0.5 * (-w.real * qx + w.imag * qy + py))


@pytest.mark.parametrize("nz", [16, 64, 400])
def test_real_transform_pre_and_post(nz):
    """Length-nz real rows as M = nz / 2 complex values: the C2R pre-processing
    followed by an inverse complex FFT of length M gives the real row, and the R2C
    post-processing of a forward complex FFT gives the half spectrum."""
    M = nz // 2
    rng = np.random.default_rng(nz)
    c = rng.standard_normal(nz)
    X = np.fft.rfft(c)  # X_0 .. X_M
    w = np.exp(-2j * np.pi * np.arange(M + 1) / nz)
    Z = np.array([c2r_pre(X[k] if k else complex(X[0].real, 0), X[M - k] if k else complex(X[M].real, 0), w[k])
                  for k in range(M)])
    z = np.fft.ifft(Z) * M  # unnormalised inverse of length M: z[m] = (c[2m] + i c[2m+1]) * nz ... scale
    got = np.empty(nz)
    got[0::2], got[1::2] = z.real, z.imag
    assert np.abs(got - c * nz).max() < 1e-10 * nz  # C2R of the full spectrum, unnormalised
    zf = np.fft.fft(c[0::2] + 1j * c[1::2])
    Xg = np.array([r2c_post(zf[k], zf[(M - k) % M], w[k]) for k in range(M)])
    assert np.abs(Xg - X[:M]).max() < 1e-10 * nz
