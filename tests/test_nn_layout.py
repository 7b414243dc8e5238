"""Index models of the surrogate kernels added for speed (host logic, no GPU).

Restated from csrc/evx_nn_tc.cu and csrc/evx_nn.cu:
  - resid32_staged: an epilogue warp stages 32 voxels x 16 channels of FP32 sums,
    16-byte chunk q of row (voxel) v at chunk q ^ ((v >> 1) & 3), written with lane = v
    and read with lane l on voxel l / 4 + 8 i, chunk l % 4;
  - project_lane_kernel / lift_lane_kernel: warp units (b, x, y0, z0) of RY = 2 rows x
    32 z, lane = channel, the 32-value butterfly that leaves lane l with the lane sum of
    value l;
  - bias_grad_vec_kernel: C / 8 threads per voxel, 16-byte pieces, the per-channel
    reduction over a CTA's threads.
"""
import numpy as np
import pytest


def wavefront_conflicts(chunk_addrs):
    """16-byte accesses are served 8 lanes (128 bytes) per wavefront: count the
    extra wavefronts caused by two lanes of a phase on the same 4-bank group."""
    extra = 0
    for p0 in range(0, len(chunk_addrs), 8):
        groups = [(a // 16) % 8 for a in chunk_addrs[p0:p0 + 8]]
        extra += len(groups) - len(set(groups))
    return extra


def test_resid32_staging_swizzle():
    floats = 32 * 16
    written = {}
    for q in range(4):  # one STS.128 per q
        addrs = []
        for lane in range(32):
            idx = lane * 16 + 4 * (q ^ ((lane >> 1) & 3))
            assert 0 <= idx and idx + 4 <= floats
            written[(lane, q)] = idx
            addrs.append(idx * 4)
        assert wavefront_conflicts(addrs) == 0
    assert len(set(written.values())) == 32 * 4  # every chunk written once
    read = set()
    for i in range(4):  # one LDS.128 per i
        addrs = []
        for lane in range(32):
            v, c = (lane >> 2) + 8 * i, lane & 3
            idx = v * 16 + 4 * (c ^ ((v >> 1) & 3))
            assert idx == written[(v, c)]  # the chunk written by lane v for channels 4c ..
            read.add((v, c))
            addrs.append(idx * 4)
        assert wavefront_conflicts(addrs) == 0
    assert len(read) == 128
    # global side: the warp's 32 voxels x 16 channels (c0 = 0 or 16), each float once,
    # 4 lanes on one 64-byte row piece
    for c0 in (0, 16):
        seen = set()
        for i in range(4):
            for lane in range(32):
                v, c = (lane >> 2) + 8 * i, lane & 3
                o = v * 32 + c0 + 4 * c
                for k in range(4):
                    assert (o + k) not in seen
                    seen.add(o + k)
        assert seen == {v * 32 + c0 + j for v in range(32) for j in range(16)}


def butterfly(V):
    v = V.copy()
    off = 16
    while off >= 1:
        new = v.copy()
        for lane in range(32):
            partner = lane ^ off
            up, pup = bool(lane & off), bool(partner & off)
            for k in range(off):
                send_p = v[partner][k] if pup else v[partner][k + off]
                keep = v[lane][k + off] if up else v[lane][k]
                new[lane][k] = keep + send_p
        v = new
        off //= 2
    return v[:, 0]


def test_lane_butterfly_sums():
    rng = np.random.default_rng(3)
    V = rng.standard_normal((32, 32))
    assert np.allclose(butterfly(V), V.sum(axis=0), rtol=0, atol=1e-12)
    # a plausible mistake (lanes keeping the other half) must fail
    W = V.copy()
    W[:, :16], W[:, 16:] = V[:, 16:], V[:, :16]
    assert not np.allclose(butterfly(W), V.sum(axis=0))


def wrapi(i, n):
    assert -n <= i < 2 * n
    return i + n if i < 0 else (i - n if i >= n else i)


@pytest.mark.parametrize("B,X,Y,Z", [(1, 1, 2, 32), (2, 3, 4, 64), (1, 2, 6, 96)])
def test_lane_units_cover_outputs(B, X, Y, Z):
    RY = 2
    nzr, nyr = Z // 32, Y // RY
    units = B * X * nyr * nzr
    seen = np.zeros((B, X, Y, Z), dtype=int)
    for u in range(units):
        z0 = (u % nzr) * 32
        r = u // nzr
        y0 = (r % nyr) * RY
        r //= nyr
        x, b = r % X, r // X
        assert b < B
        for ry in range(RY):
            seen[b, x, y0 + ry, z0:z0 + 32] += 1
        # inputs: rows y0 - 1 .. y0 + RY, x +- 1, z0 - 1 .. z0 + 32 with periodic wrap
        for yy in range(RY + 2):
            assert 0 <= wrapi(y0 + yy - 1, Y) < Y
        for dx in range(3):
            assert 0 <= wrapi(x + dx - 1, X) < X
        assert 0 <= wrapi(z0 - 1, Z) < Z and 0 <= wrapi(z0 + 32, Z) < Z
        for lane in range(32):  # the lift's shuffled loads
            assert 0 <= wrapi(z0 - 1 + lane, Z) < Z
            if lane < 2:
                assert 0 <= wrapi(z0 + 31 + lane, Z) < Z
    assert (seen == 1).all()


@pytest.mark.parametrize("C", [16, 32])
def test_bias_grad_vec_mapping(C):
    TPV, NT = C // 8, 256
    for nblocks, nvox in [(3, 100), (304, 5000), (2, 1)]:
        stride = nblocks * NT // TPV
        hits = np.zeros((nvox, C), dtype=int)
        for blk in range(nblocks):
            for t in range(NT):
                piece = t % TPV
                v = (blk * NT + t) // TPV
                while v < nvox:
                    for u in range(4):
                        vu = v + u * stride
                        if vu < nvox:
                            hits[vu, 8 * piece:8 * piece + 8] += 1
                    v += 4 * stride
        assert (hits == 1).all()
        # the CTA reduction: thread co < C sums red[t][co % 8] over t = co / 8 (mod TPV)
        for co in range(C):
            ts = list(range(co // 8, NT, TPV))
            assert all(t % TPV == co // 8 for t in ts) and len(ts) == NT // TPV
