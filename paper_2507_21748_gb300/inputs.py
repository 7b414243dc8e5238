"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds only random-number generation and the input recipes; none
of the method's arithmetic. Every field is produced on the host in FP64 and
rounded to FP32 before either side sees it, so a comparison measures the
solver, not the rounding of its input.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used as a counter-based generator. For seed
s and linear voxel index i (C order, z fastest) the state is
    x = s * 0x9E3779B97F4A7C15 + i          (mod 2^64)
and the draw is the SplitMix64 output for that state:
    z = x + 0x9E3779B97F4A7C15
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    z =  z ^ (z >> 31)
    u = (z >> 11) / 2^53                      in [0, 1)
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_uniform(seed: int, start: int, count: int) -> np.ndarray:
    """u_i in [0,1) (float64) for i = start .. start+count-1."""
    with np.errstate(over="ignore"):
        i = np.arange(start, start + count, dtype=np.uint64)
        x = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GAMMA + i
        z = x + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_field(shape, seed=0, lo=-0.05, hi=0.05, offset=0.0, chunk=1 << 24) -> np.ndarray:
    """offset + U(lo, hi) i.i.d. per voxel, computed in FP64, returned as float32."""
    n = int(np.prod(shape))
    out = np.empty(n, dtype=np.float32)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        u = splitmix64_uniform(seed, s, m)
        out[s:s + m] = (offset + lo + (hi - lo) * u).astype(np.float32)
    return out.reshape(shape)


def mode_field(shape, terms, offset=0.0) -> np.ndarray:
    """offset + sum_j A_j cos(2 pi (m_j . x / N) + phase_j), float32.

    terms: iterable of (A, (mx, my, mz), phase)."""
    nx, ny, nz = shape
    x = np.arange(nx)[:, None, None] / nx
    y = np.arange(ny)[None, :, None] / ny
    z = np.arange(nz)[None, None, :] / nz
    f = np.full(shape, float(offset), dtype=np.float64)
    for A, (mx, my, mz), ph in terms:
        f = f + A * np.cos(2 * np.pi * (mx * x + my * y + mz * z) + ph)
    return f.astype(np.float32)


def trajectory_mean(seed: int, lo=-0.3, hi=0.3) -> float:
    """Mean composition of training trajectory ``seed`` (surrogate data set):
    drawn from the same generator with the seed's stream offset past any grid."""
    u = splitmix64_uniform(seed, 1 << 62, 1)[0]
    return float(np.float32(lo + (hi - lo) * u))
