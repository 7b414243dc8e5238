"""Host model of the fused y-z-y pass (csrc/evx_fused.cu): its work schedule,
shared-memory layout and global index ranges, checked on the CPU for every
geometry the dispatch instantiates (no GPU).

Restated rules:
  - items per x slab: Yinv and Yfwd one per chunk of 8 columns (Zp / 8 chunks),
    Z one per RPC = 8 TPy / TPz consecutive rows (ny / RPC items);
  - ticket t: phase p = t // per, offset o = t % per, per = 2 chunks + z items;
    o < chunks: Yinv(slab p); then Z(slab p - lag); then Yfwd(slab p - 2 lag);
  - a Z item of slab x waits for all Yinv items of x, a Yfwd item for all Z items;
  - element (x, y, kz) at ((y // YB) nx + x) YB + y % YB) Zp + kz;
  - one shared tile buffer of max((L + TPy) 8, RPC BS [+ RPC zxs]) float2, then
    the twiddle tables.
"""
import random

import numpy as np
import pytest

from test_fast_layout import slot, zpad, zxs

# (ny = L, R1y, TPy, M, R1z, TPz, YB)
GEOMS = [(1024, 32, 32, 512, 32, 16, 32), (512, 32, 16, 256, 32, 8, 32), (256, 32, 8, 128, 32, 4, 32),
         (400, 20, 20, 200, 20, 10, 16)]
SMEM_MAX = 227 * 1024


def geom(L, R1y, TPy, M, R1z, TPz):
    NT = 8 * TPy
    RPC = NT // TPz
    Zp = ((M + 1 + 7) // 8) * 8
    RS = M + TPz * zpad(R1z, TPz)
    BS = TPz + ((max(Zp, RS) - TPz + 15) & ~15)
    YT = (L + TPy) * 8
    ZT = RPC * BS + (RPC * zxs(M, TPz) if R1z != 32 else 0)
    tile = max(YT, ZT)
    YTW = L if R1y == TPy else 2 * L
    floats2 = tile + YTW + 3 * M + 1
    return dict(NT=NT, RPC=RPC, Zp=Zp, BS=BS, YT=YT, ZT=ZT, tile=tile, YTW=YTW, floats2=floats2)


def decode(t, per, nyi, nzi, lag):
    ph, o = divmod(t, per)
    if o < nyi:
        return 0, ph, o
    if o < nyi + nzi:
        return 1, ph - lag, o - nyi
    return 2, ph - 2 * lag, o - nyi - nzi


@pytest.mark.parametrize("g", GEOMS)
def test_shared_memory_layout(g):
    L, R1y, TPy, M, R1z, TPz, YB = g
    G = geom(L, R1y, TPy, M, R1z, TPz)
    NT, RPC, BS = G["NT"], G["RPC"], G["BS"]
    assert NT % 32 == 0 and NT % TPz == 0 and YB % RPC == 0 and L % RPC == 0
    assert G["floats2"] * 8 <= SMEM_MAX
    # y item: loads/stores in 16-byte pieces, the padded transpose, the row-order staging
    for t in range(NT):
        p, n2 = t & 7, t >> 3
        assert n2 < TPy
        for n1 in range(R1y):
            assert (n2 + TPy * n1) * 8 + p < G["YT"]
        for a in range(R1y):
            assert slot(R1y, TPy, 8, 1, n2, a, p) < G["YT"]
        NB = R1y // TPy
        for i in range(NB):
            for c in range(TPy):
                assert slot(R1y, TPy, 8, 1, c, n2 * NB + i, p) < G["YT"]
                assert (n2 * NB + i + R1y * c) * 8 + p < L * 8
    for e in range(L * 4):
        y, q = e >> 2, e & 3
        assert y * 8 + 2 * q + 1 < L * 8 and (y * 8 + 2 * q) % 2 == 0
    # z item: row loads, both transposes, partner rows beyond the rows
    pad, NBz = zpad(R1z, TPz), R1z // TPz
    Zh = G["Zp"] // 2
    for e in range(RPC * Zh):
        rr, q = divmod(e, Zh)
        assert rr * BS + 2 * q + 1 < RPC * BS
    for t in range(NT):
        n2, r = t % TPz, t // TPz
        for a in range(R1z):
            assert r * BS + slot(R1z, TPz, 1, pad, n2, a, 0) < (r + 1) * BS
        for i in range(NBz):
            for c in range(TPz):
                assert r * BS + slot(R1z, TPz, 1, pad, c, n2 * NBz + i, 0) < (r + 1) * BS
        if R1z != 32:
            for d in range(R1z):
                assert RPC * BS + r * zxs(M, TPz) + n2 + TPz * d < G["ZT"]
    assert G["ZT"] <= G["tile"] and G["YT"] <= G["tile"]


@pytest.mark.parametrize("g", GEOMS)
@pytest.mark.parametrize("nx", [3, 24])
def test_items_cover_each_element_once(g, nx):
    L, R1y, TPy, M, R1z, TPz, YB = g
    G = geom(L, R1y, TPy, M, R1z, TPz)
    ny, Zp, RPC = L, G["Zp"], G["RPC"]
    ncols, nch = M + 1, Zp // 8
    os2, xs = nx * YB * Zp, YB * Zp
    total = nx * ny * Zp
    # y items: (x, chunk) x (y, q) pieces of nval valid columns
    x, chunk, y, q = np.meshgrid(np.arange(nx), np.arange(nch), np.arange(ny), np.arange(4), indexing="ij")
    kz = chunk * 8 + 2 * q
    nval = np.clip(ncols - kz, 0, 2)
    off = x * xs + (y // YB) * os2 + (y % YB) * Zp + kz
    seen = np.zeros(total, dtype=np.int64)
    for j in (0, 1):
        m = nval > j
        assert (off[m] + j < total).all()
        np.add.at(seen, (off[m] + j).ravel(), 1)
    want = np.tile((np.arange(Zp) < ncols).astype(np.int64), nx * ny)
    assert np.array_equal(seen, want)
    # z items: RPC consecutive memory rows inside one y block
    xx, idx = np.meshgrid(np.arange(nx), np.arange(ny // RPC), indexing="ij")
    y0 = RPC * idx
    assert ((y0 % YB) + RPC <= YB).all()
    r0 = ((y0 // YB) * nx + xx) * YB + y0 % YB
    rows = (r0[..., None] + np.arange(RPC)).ravel()
    assert rows.max() < nx * ny
    assert np.array_equal(np.bincount(rows, minlength=nx * ny), np.ones(nx * ny, dtype=np.int64))


@pytest.mark.parametrize("g", GEOMS)
@pytest.mark.parametrize("nx,lag", [(8, 1), (24, 3), (64, 3), (16, 16)])
def test_ticket_order_dependencies_and_progress(g, nx, lag):
    """Every dependency has a lower ticket, each slab's counters reach exactly their
    targets, and a simulated run with fewer workers than items (random item times,
    a worker blocks while its item waits) finishes."""
    L, R1y, TPy, M, R1z, TPz, YB = g
    G = geom(L, R1y, TPy, M, R1z, TPz)
    nyi, nzi = G["Zp"] // 8, L // G["RPC"]
    per = 2 * nyi + nzi
    total = (nx + 2 * lag) * per
    first = {}
    last = {}
    count = {}
    for t in range(total):
        k, x, i = decode(t, per, nyi, nzi, lag)
        if not 0 <= x < nx:
            continue
        first.setdefault((k, x), t)
        last[(k, x)] = t
        count[(k, x)] = count.get((k, x), 0) + 1
    for x in range(nx):
        assert count[(0, x)] == nyi and count[(1, x)] == nzi and count[(2, x)] == nyi
        assert last[(0, x)] < first[(1, x)] and last[(1, x)] < first[(2, x)]
    # simulation: W workers take tickets in order; an item runs once its slab's previous stage is done
    rng = random.Random(1)
    W = 37
    done = {}
    clock = 0.0
    finish = [0.0] * W
    nxt = 0
    cnt = {}
    busy = []  # (finish time, worker, item)
    free = list(range(W))
    pending = []  # (worker, item) waiting on a dependency
    while nxt < total or busy or pending:
        while free and nxt < total:
            w = free.pop()
            item = decode(nxt, per, nyi, nzi, lag)
            nxt += 1
            if not 0 <= item[1] < nx:
                free.append(w)
                continue
            pending.append((w, item))
        progressed = True
        while progressed:
            progressed = False
            for w, item in list(pending):
                k, x, _ = item
                need = {0: None, 1: ((0, x), nyi), 2: ((1, x), nzi)}[k]
                if need is None or cnt.get(need[0], 0) >= need[1]:
                    pending.remove((w, item))
                    busy.append((clock + rng.uniform(0.5, 2.0), w, item))
                    progressed = True
        assert busy, "deadlock"
        busy.sort()
        t_end, w, item = busy.pop(0)
        clock = t_end
        cnt[(item[0], item[1])] = cnt.get((item[0], item[1]), 0) + 1
        free.append(w)
    assert all(cnt[(2, x)] == nyi for x in range(nx))
