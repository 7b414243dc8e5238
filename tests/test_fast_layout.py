"""Shared-memory layout model of the fast step kernels (host logic, no GPU).

The index rules of csrc/evx_fast.cu are restated here and every thread's shared-
memory index is enumerated for each instantiation the dispatch uses. The tests
check that each index stays inside its buffer, and that accesses the design calls
conflict-free put the 16 threads of a half-warp (one 128-byte wavefront of float2)
on 16 distinct bank pairs.
  - transposes: slot(n2, a, p) = (a TP + n2 + (a / NB) pad) P + p, NB = R1 / TP
  - z-pass pad: the smallest d with s = R1 + d odd and (s - 1) TP = 0 (mod 16)
  - z-pass tile rows: BS = TP + roundup16(max(Zp, M + TP pad) - TP), = TP (mod 16)
  - z-pass partner rows: stride M rounded up to = TP (mod 16)
"""
import pytest


def zpad(R1, TP):
    for d in range(1, 16):
        if ((R1 + d) & 1) and ((R1 + d - 1) * TP) % 16 == 0:
            return d
    return 1


def zxs(M, TP):
    return M + (((TP - M) % 16) + 16) % 16


def xbox(L):
    return L if L <= 256 else (256 if L % 256 == 0 else L // 2)


def slot(R1, TP, P, pad, n2, a, p):
    NB = R1 // TP
    return (a * TP + n2 + a // NB * pad) * P + p


def distinct_pairs(addrs):
    """extra threads sharing a bank pair (float2 index mod 16) in one half-warp"""
    return len(addrs) - len({x % 16 for x in addrs})


# (R1, TP) of every x / y pass the dispatch instantiates, and of every z pass (M = nz / 2)
XY = [(32, 2), (32, 4), (32, 8), (32, 16), (32, 32), (20, 20)]
Z = [(32, 2, 128), (32, 4, 128), (32, 8, 128), (32, 16, 128), (20, 10, 160)]


@pytest.mark.parametrize("R1,TP", XY)
def test_strided_pass_layout(R1, TP):
    """x and y passes (8 columns per tile, 8 TP threads, p fastest)."""
    P, L, NB = 8, R1 * TP, R1 // TP
    XB = (L + TP) * P
    assert L % xbox(L) == 0 and xbox(L) <= 256
    assert (XB * 8) % 128 == 0 and (xbox(L) * P * 8) % 128 == 0  # TMA destinations stay 128-byte aligned
    extra = 0
    threads = range(P * TP)
    for t in threads:
        p, n2 = t % P, t // P
        for n1 in range(R1):
            assert (n2 + TP * n1) * P + p < L * P  # tile loads and the store staging
        for a in range(R1):
            assert slot(R1, TP, P, 1, n2, a, p) < XB
        for i in range(NB):
            for c in range(TP):
                assert slot(R1, TP, P, 1, c, n2 * NB + i, p) < XB
                assert n2 * NB + i + R1 * c < L  # |k_x|^2 index
    for h0 in range(0, P * TP, 16):
        hw = range(h0, min(h0 + 16, P * TP))
        for a in range(R1):
            extra += distinct_pairs([slot(R1, TP, P, 1, t // P, a, t % P) for t in hw])
        for i in range(NB):
            for c in range(TP):
                extra += distinct_pairs([slot(R1, TP, P, 1, c, (t // P) * NB + i, t % P) for t in hw])
    assert extra == 0


@pytest.mark.parametrize("R1,TP,NTZ", Z)
def test_z_pass_layout(R1, TP, NTZ):
    """z pass: RPC = NTZ / TP rows of TP threads; both transposes and the partner rows."""
    M, NB, RPC = R1 * TP, R1 // TP, NTZ // TP
    pad = zpad(R1, TP)
    Zp = ((M + 1 + 7) // 8) * 8
    RS = M + TP * pad
    BS = TP + ((max(Zp, RS) - TP + 15) & ~15)
    XS = zxs(M, TP)
    assert NTZ % TP == 0 and NTZ % 32 == 0 and BS % 16 == TP % 16 and BS % 2 == 0
    if R1 == 32:
        assert pad == 1  # the power-of-two kernels keep the one-group pad
    for rr in range(RPC):
        for q in range(max(Zp // 2, M // 2)):
            assert rr * BS + 2 * q + 1 < RPC * BS  # 16-byte row loads / stores
    extra = 0
    for t in range(NTZ):
        n2, r = t % TP, t // TP
        for n1 in range(R1):
            k = n2 + TP * n1
            assert k < M and M - k < Zp  # C2R pre-processing reads X_k and X_{M-k}
        for a in range(R1):
            assert 0 <= slot(R1, TP, 1, pad, n2, a, 0) < BS
        for i in range(NB):
            for c in range(TP):
                assert 0 <= slot(R1, TP, 1, pad, c, n2 * NB + i, 0) < BS
                assert n2 * NB + i + R1 * c < M  # real-row staging (float2 index < nz / 2)
        for d in range(R1):
            assert n2 + TP * d < M <= XS
    for h0 in range(0, NTZ, 16):
        hw = range(h0, h0 + 16)
        for a in range(R1):
            extra += distinct_pairs([(t // TP) * BS + slot(R1, TP, 1, pad, t % TP, a, 0) for t in hw])
        for i in range(NB):
            for c in range(TP):
                extra += distinct_pairs([(t // TP) * BS + slot(R1, TP, 1, pad, c, (t % TP) * NB + i, 0) for t in hw])
        if R1 != 32:
            for d in range(R1):
                extra += distinct_pairs([(t // TP) * XS + t % TP + TP * d for t in hw])
    assert extra == 0


def test_z_pass_pad_one_conflicts_for_ten_thread_pencils():
    """The one-group pad of the power-of-two kernels is not enough for TP = 10: block
    ownership then puts two threads of a half-warp on one bank pair."""
    R1, TP, NTZ = 20, 10, 160
    M, NB = R1 * TP, R1 // TP
    BS = TP + ((max(208, M + TP) - TP + 15) & ~15)
    extra = 0
    for h0 in range(0, NTZ, 16):
        hw = range(h0, h0 + 16)
        for i in range(NB):
            for c in range(TP):
                extra += distinct_pairs([(t // TP) * BS + slot(R1, TP, 1, 1, c, (t % TP) * NB + i, 0) for t in hw])
    assert extra > 0
