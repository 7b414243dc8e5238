"""GPU kernels of the learned surrogate against the FP64 oracle (oracle/nn.py).

Inputs and weights are rounded to BF16 once and given to both sides, so the
comparison measures the kernels (FP32 accumulation, BF16 outputs), not the
input rounding."""
import numpy as np
import pytest

from oracle import nn as N

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_21748_gb300 import surrogate
    return surrogate


def bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


SHAPE = (2, 4, 6, 64)  # B, X, Y, Z


@pytest.mark.parametrize("cin,cout", [(16, 32), (32, 32), (32, 16), (16, 16)])
@pytest.mark.parametrize("epi", [0, 1, 2, 3, 4])
def test_conv_forward_epilogues(S, cin, cout, epi):
    import torch
    rng = np.random.default_rng(cin * 100 + cout + epi)
    x = bf16(rng.standard_normal(SHAPE + (cin,)))
    w = bf16(rng.standard_normal((27, cout, cin)) * 0.1)
    b = torch.from_numpy(rng.standard_normal(cout).astype(np.float32))
    pre = bf16(rng.standard_normal(SHAPE + (cout,)))
    res = bf16(rng.standard_normal(SHAPE + (cout,)))
    xd, wd, bd, pred_, resd = x.cuda(), w.cuda(), b.cuda(), pre.cuda(), res.cuda()
    if epi == 4:
        out = torch.empty(SHAPE, dtype=torch.float32, device="cuda")
    else:
        out = torch.empty(SHAPE + (cout,), dtype=torch.bfloat16, device="cuda")
    B, X, Y, Z = SHAPE
    S._ck(S.lib.evx_nn_conv3d(S._p(xd), S._p(wd), S._p(bd), S._p(out), S._p(pred_), S._p(resd),
                              B, X, Y, Z, cin, cout, epi, S._stream()))
    torch.cuda.synchronize()
    ref = N.conv(x.float().numpy().astype(np.float64), w.float().numpy().astype(np.float64),
                 b.numpy().astype(np.float64))
    got = out.float().cpu().numpy()
    if epi == 4:
        assert rel(got, ref[..., 0]) < 1e-5
        return
    if epi == 1:
        assert rel(pred_.float().cpu().numpy(), ref) < 8e-3
        ref = N.gelu(ref)
    elif epi == 2:
        ref = ref + res.float().numpy()
    elif epi == 3:
        ref = ref * N.gelu_grad(pre.float().numpy().astype(np.float64))
    assert rel(got, ref) < 8e-3  # BF16 output rounding (2^-9 relative)


def _conv32(S, engine, shape, epi, seed):
    import torch
    rng = np.random.default_rng(seed)
    x = bf16(rng.standard_normal(shape + (32,)))
    w = bf16(rng.standard_normal((27, 32, 32)) * 0.1)
    b = torch.from_numpy(rng.standard_normal(32).astype(np.float32))
    pre = bf16(rng.standard_normal(shape + (32,)))
    res = bf16(rng.standard_normal(shape + (32,)))
    xd, wd, bd, pred_, resd = x.cuda(), w.cuda(), b.cuda(), pre.cuda(), res.cuda()  # held until the check
    out = torch.empty(shape + (32,), dtype=torch.bfloat16, device="cuda")
    B, X, Y, Z = shape
    S.set_conv_engine(engine)
    try:
        S._ck(S.lib.evx_nn_conv3d(S._p(xd), S._p(wd), S._p(bd), S._p(out), S._p(pred_), S._p(resd),
                                  B, X, Y, Z, 32, 32, epi, S._stream()))
        S.check()
    finally:
        S.set_conv_engine(S.ENGINE_TCGEN05)
    ref = N.conv(x.float().numpy().astype(np.float64), w.float().numpy().astype(np.float64),
                 b.numpy().astype(np.float64))
    if epi == 1:
        assert rel(pred_.float().cpu().numpy(), ref) < 8e-3
        ref = N.gelu(ref)
    elif epi == 2:
        ref = ref + res.float().numpy()
    elif epi == 3:
        ref = ref * N.gelu_grad(pre.float().numpy().astype(np.float64))
    return out.float().cpu().numpy(), ref


@pytest.mark.parametrize("shape", [(1, 3, 4, 64), (2, 2, 2, 128), (1, 5, 6, 192), (1, 1, 2, 64), (1, 3, 16, 128),
                                   (1, 2, 50, 128), (2, 3, 4, 256)])
@pytest.mark.parametrize("epi", [0, 1, 2, 3])
def test_conv32_engines_agree_with_oracle(S, shape, epi):
    """32 -> 32 convolution on the tcgen05 engine and on the mma.sync engine:
    both within BF16 output rounding of the FP64 oracle, and within a few BF16
    ulps of each other (same BF16 operands, FP32 accumulation in another order).
    Z a multiple of 128 takes the pipelined kernel (Y = 16 and 50 split the
    columns into y segments, 50 into ragged ones), other Z the tile kernel;
    X = 1 and Y = 2 make periodic neighbours wrap onto the tile itself."""
    seed = sum(shape) * 10 + epi
    got_tc, ref = _conv32(S, S.ENGINE_TCGEN05, shape, epi, seed)
    got_ms, _ = _conv32(S, S.ENGINE_MMA_SYNC, shape, epi, seed)
    assert rel(got_tc, ref) < 8e-3
    assert rel(got_ms, ref) < 8e-3
    assert rel(got_tc, got_ms) < 8e-3
    assert np.max(np.abs(got_tc - ref)) < 0.05 * np.max(np.abs(ref)) + 0.05


def test_conv_engine_setting(S):
    import paper_2507_21748_gb300.evx as evx
    assert S.conv_engine() == S.ENGINE_TCGEN05
    with pytest.raises(evx.EvxError):
        S.set_conv_engine(7)
    S.set_conv_engine(S.ENGINE_MMA_SYNC)
    assert S.conv_engine() == S.ENGINE_MMA_SYNC
    S.set_conv_engine(S.ENGINE_TCGEN05)
    S.check()


@pytest.mark.parametrize("shape", [(2, 4, 6, 64), (1, 3, 5, 7), (1, 1, 1, 9), (1, 1, 2, 32), (3, 2, 4, 96)])
def test_direct_lift_and_projection(S, shape):
    """evx_nn_lift and evx_nn_project against the FP64 oracle's conv on the padded
    input / channel 0 of the output, and against the tensor-core convolutions
    they replace (same BF16 operands: FP32 sums in another order); any sizes,
    periodic (X = Y = 1 wraps every neighbour onto the voxel's own row)."""
    import torch
    rng = np.random.default_rng(sum(shape))
    B, X, Y, Z = shape
    f = rng.standard_normal(shape).astype(np.float32)
    w0 = rng.standard_normal((27, 32, 16)) * 0.2
    w0[:, :, 1:] = 0.0
    w0 = bf16(w0)
    b0 = torch.from_numpy(rng.standard_normal(32).astype(np.float32))
    fd, w0d, b0d = torch.from_numpy(f).cuda(), w0.cuda(), b0.cuda()
    h = torch.empty(shape + (32,), dtype=torch.bfloat16, device="cuda")
    S._ck(S.lib.evx_nn_lift(S._p(fd), 1.0, S._p(w0d), 16, 32, S._p(b0d), S._p(h), B, X, Y, Z, S._stream()))
    wp = bf16(rng.standard_normal((27, 16, 32)) * 0.1)
    bp = torch.from_numpy(rng.standard_normal(16).astype(np.float32))
    hin = bf16(rng.standard_normal(shape + (32,)))
    hd, wpd, bpd = hin.cuda(), wp.cuda(), bp.cuda()
    d = torch.empty(shape, dtype=torch.float32, device="cuda")
    S._ck(S.lib.evx_nn_project(S._p(hd), S._p(wpd), 32, 16, S._p(bpd), S._p(d), B, X, Y, Z, S._stream()))
    torch.cuda.synchronize()
    a_in = N.field_to_act(bf16(f).float().numpy().astype(np.float64))
    ref_h = N.conv(a_in, w0.float().numpy().astype(np.float64), b0.numpy().astype(np.float64))
    assert rel(h.float().cpu().numpy(), ref_h) < 8e-3  # BF16 output rounding
    ref_d = N.conv(hin.float().numpy().astype(np.float64), wp.float().numpy().astype(np.float64),
                   bp.numpy().astype(np.float64))[..., 0]
    assert rel(d.cpu().numpy(), ref_d) < 1e-5  # FP32 output
    if Z % 64 == 0 and Y % 2 == 0:  # the tensor-core path these replace
        act = torch.empty(shape + (16,), dtype=torch.bfloat16, device="cuda")
        S._ck(S.lib.evx_nn_field_to_act(S._p(fd), B * X * Y * Z, 16, 1.0, S._p(act), S._stream()))
        h2 = torch.empty_like(h)
        S._ck(S.lib.evx_nn_conv3d(S._p(act), S._p(w0d), S._p(b0d), S._p(h2), None, None, B, X, Y, Z, 16, 32, 0,
                                  S._stream()))
        d2 = torch.empty_like(d)
        S._ck(S.lib.evx_nn_conv3d(S._p(hd), S._p(wpd), S._p(bpd), S._p(d2), None, None, B, X, Y, Z, 32, 16, 4,
                                  S._stream()))
        torch.cuda.synchronize()
        assert rel(h.float().cpu().numpy(), h2.float().cpu().numpy()) < 8e-3
        assert rel(d.cpu().numpy(), d2.cpu().numpy()) < 1e-5


@pytest.mark.parametrize("cin,cout", [(16, 32), (32, 32), (32, 16)])
def test_conv_dgrad_and_wgrad(S, cin, cout):
    import torch
    rng = np.random.default_rng(7 + cin + cout)
    x = bf16(rng.standard_normal(SHAPE + (cin,)))
    dy = bf16(rng.standard_normal(SHAPE + (cout,)))
    w = bf16(rng.standard_normal((27, cout, cin)) * 0.1)
    B, X, Y, Z = SHAPE
    xd, dyd, wd = x.cuda(), dy.cuda(), w.cuda()
    wt = torch.empty((27, cin, cout), dtype=torch.bfloat16, device="cuda")
    S._ck(S.lib.evx_nn_flip_weights(S._p(wd), cout, cin, S._p(wt), S._stream()))
    dx = torch.empty(SHAPE + (cin,), dtype=torch.bfloat16, device="cuda")
    S._ck(S.lib.evx_nn_conv3d(S._p(dyd), S._p(wt), None, S._p(dx), None, None, B, X, Y, Z, cout, cin, 0,
                              S._stream()))
    dw = torch.empty((27, cout, cin), dtype=torch.float32, device="cuda")
    part = torch.empty(64 * 27 * cin * cout, dtype=torch.float32, device="cuda")
    S._ck(S.lib.evx_nn_conv3d_wgrad(S._p(dyd), S._p(xd), S._p(dw), S._p(part), part.numel(), B, X, Y, Z, cin,
                                    cout, S._stream()))
    torch.cuda.synchronize()
    xn, dyn, wn = (t.float().numpy().astype(np.float64) for t in (x, dy, w))
    assert rel(dx.float().cpu().numpy(), N.conv_dgrad(dyn, wn)) < 8e-3
    assert rel(dw.cpu().numpy(), N.conv_wgrad(dyn, xn)) < 1e-5


def test_network_forward_and_gradients_vs_oracle(S):
    import torch
    shape, B = (6, 4, 64), 2
    net = S.Net(shape, B, seed=3)
    # a net whose blocks do something: larger second convs and projection
    rng = np.random.default_rng(4)
    for n in net.names:
        if n.startswith("W2_") or n == "Wp":
            net.p[n].mul_(10.0 if n != "Wp" else 30.0)
        if n.startswith("b"):
            net.p[n].copy_(torch.from_numpy(rng.standard_normal(net.p[n].shape).astype(np.float32) * 0.05))
    net.p["Wp"][:, 1:, :] = 0
    net.p["bp"][1:] = 0
    net._refresh_bf16()
    c = rng.uniform(-0.4, 0.4, (B,) + shape).astype(np.float32)
    t = (c + rng.normal(0, 0.05, c.shape)).astype(np.float32)
    cd, td = torch.from_numpy(c).cuda(), torch.from_numpy(t).cuda()
    pred = net.forward(cd).clone()
    L = net.backward(td)
    torch.cuda.synchronize()
    P = net.params_numpy()
    Lr, pr, gr = N.loss_and_grads(P, c.astype(np.float64), t.astype(np.float64))
    assert rel(pred.cpu().numpy() - c, pr - c) < 2e-2
    assert abs(L - Lr) < 2e-2 * Lr
    # mass: the correction is zero-mean per sample (FP64 mean, FP32 field)
    drift = np.abs((pred.cpu().numpy().astype(np.float64) - c).sum(axis=(1, 2, 3)))
    assert drift.max() < 1e-6 * np.abs(c).sum(axis=(1, 2, 3)).min()
    flat = {"W0": gr["W0"], "b0": gr["b0"], "Wp": gr["Wp"], "bp": gr["bp"]}
    for k, (dW1, db1, dW2, db2) in enumerate(gr["blocks"]):
        flat.update({"W1_%d" % k: dW1, "b1_%d" % k: db1, "W2_%d" % k: dW2, "b2_%d" % k: db2})
    scale = max(float(np.abs(r).max()) for r in flat.values())
    for n, ref in flat.items():
        got = net.g[n].cpu().numpy().astype(np.float64)
        if n in ("Wp", "bp"):
            got, ref = got[:, :1] if n == "Wp" else got[:1], ref[:, :1] if n == "Wp" else ref[:1]
        if n == "W0":
            got, ref = got[..., :1], ref[..., :1]
        if np.abs(ref).max() < 1e-9 * scale:
            # a parameter that only adds a constant to the correction (the projection
            # bias, the last block's output bias): zero-mean output makes its exact
            # gradient 0; the GPU returns the rounding noise of a BF16 sum
            assert np.abs(got).max() < 1e-3 * scale, n
            continue
        cos = float(np.sum(got * ref) / (np.linalg.norm(got) * np.linalg.norm(ref) + 1e-300))
        assert cos > 0.999 and rel(got, ref) < 5e-2, (n, cos, rel(got, ref))


def test_training_beats_persistence_and_untrained(S):
    """The trained surrogate (solver-generated pairs, 10 steps per block) predicts
    held-out 10-step blocks better than c_{n+10} = c_n and than its initial state."""
    import torch
    shape, B = (32, 32, 64), 4
    pool = S.TrajectoryPool(shape, B, block=10, horizon=100, seeds=range(0, 64))
    net = S.Net(shape, B, seed=0)
    held = S.TrajectoryPool(shape, B, block=10, horizon=100, seeds=range(200, 204))
    xs, ys = [], []
    for _ in range(5):
        x, y = held.draw()
        xs.append(x.clone())
        ys.append(y.clone())

    def err(n):
        e = []
        for x, y in zip(xs, ys):
            p = n.forward(x.contiguous())
            e.append(float(((p - y) ** 2).sum() / ((y - y.mean()) ** 2).sum()) ** 0.5)
        return float(np.mean(e))

    persist = float(np.mean([float(((x - y) ** 2).sum() / ((y - y.mean()) ** 2).sum()) ** 0.5
                             for x, y in zip(xs, ys)]))
    e0 = err(net)
    # at lr 2e-3 -> 2e-4 these 300 steps are chaotic (held-out error 0.09 .. 0.52 of
    # persistence over six network seeds, and rounding-level changes in the forward
    # pass move a seed across that range); at 1e-3 -> 1e-4 every seed reached
    # 0.037 .. 0.047 on the GB300
    hist = S.train(net, pool, 300, lr=1e-3, lr_final=1e-4)
    e1 = err(net)
    pool.close()
    held.close()
    assert hist[-1] < 0.2 * hist[0]
    assert e1 < 0.2 * persist and e1 < 0.2 * e0, (e1, persist, e0)


class _Perturbed:
    """Stand-in surrogate for testing the guards: c + a fixed perturbation."""

    def __init__(self, kind, shape, B):
        import torch
        g = torch.Generator(device="cuda").manual_seed(5)
        if kind == "noise":  # large independent noise: raises the energy
            self.delta = 0.5 * torch.randn((B,) + shape, generator=g, device="cuda")
            self.delta -= self.delta.mean(dim=(1, 2, 3), keepdim=True)
        else:  # a constant: changes the mass
            self.delta = torch.full((B,) + shape, 1e-3, device="cuda")

    def forward(self, c):
        return c + self.delta


@pytest.mark.parametrize("kind", ["noise", "mass"])
def test_guarded_rollout_falls_back(S, kind):
    """A block whose prediction raises the energy or moves the mass is recomputed by
    the solver, so such a rollout equals the plain solver run (up to the FP32
    round trip of the field between blocks)."""
    import torch
    from paper_2507_21748_gb300 import inputs
    shape, B = (16, 16, 64), 2
    c0 = torch.stack([torch.from_numpy(inputs.uniform_field(shape, seed=s, offset=0.2)) for s in range(B)]).cuda()
    out, st = S.rollout(_Perturbed(kind, shape, B), c0, nblocks=3)
    ref = S.solver_run(c0, 30)
    assert st["fallbacks"] == st["blocks"] == 6
    assert rel(out.cpu().numpy(), ref.cpu().numpy().astype(np.float64)) < 1e-5


def test_guarded_rollout_accepts_the_solver_itself(S):
    """A stand-in that returns the solver's own block passes both guards."""
    import torch
    from paper_2507_21748_gb300 import inputs
    shape, B = (16, 16, 64), 2

    class Exact:
        def forward(self, c):
            return S.solver_run(c.contiguous(), 10)

    c0 = torch.stack([torch.from_numpy(inputs.uniform_field(shape, seed=s)) for s in range(B)]).cuda()
    out, st = S.rollout(Exact(), c0, nblocks=2)
    assert st["fallbacks"] == 0


def test_nonlinearity_scale_and_scaled_zero_mean_add(S):
    """evx_nn_nl_scale against its definition in FP64 (scale = min(1, ||N|| / ||d||),
    d = c - mean c, N = d^2 (3 mean + d)), and the scaled zero-mean correction."""
    import torch
    rng = np.random.default_rng(7)
    B, V = 3, 4096
    c = np.stack([0.2 + 0.05 * rng.standard_normal(V), -0.1 + 0.6 * rng.standard_normal(V),
                  np.full(V, 0.4)]).astype(np.float32)
    cd = torch.from_numpy(c).cuda()
    nparts = 8
    parts = torch.empty(3 * B * nparts, dtype=torch.float64, device="cuda")
    scale = torch.empty(B, dtype=torch.float64, device="cuda")
    S._ck(S.lib.evx_nn_nl_scale(S._p(cd), B, V, S._p(parts), nparts, S._p(scale), S._stream()))
    want = []
    for s in range(B):
        x = c[s].astype(np.float64)
        d = x - x.mean()
        N = d * d * (3 * x.mean() + d)
        want.append(min(1.0, float(np.sqrt((N * N).sum() / (d * d).sum()))) if (d * d).sum() > 0 else 0.0)
    got = scale.cpu().numpy()
    assert np.allclose(got, want, rtol=1e-9, atol=1e-12), (got, want)
    base = torch.from_numpy(rng.standard_normal((B, V)).astype(np.float32)).cuda()
    dd = torch.from_numpy(rng.standard_normal((B, V)).astype(np.float32)).cuda()
    out = torch.empty_like(base)
    dparts = torch.empty(B * nparts, dtype=torch.float64, device="cuda")
    S._ck(S.lib.evx_nn_zero_mean_add_scaled(S._p(base), S._p(dd), S._p(scale), B, V, S._p(dparts), nparts,
                                             S._p(out), S._stream()))
    dn = dd.cpu().numpy().astype(np.float64)
    ref = base.cpu().numpy() + np.array(want)[:, None] * (dn - dn.mean(axis=1, keepdims=True))
    assert np.abs(out.cpu().numpy() - ref).max() < 1e-5


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("shape", [(2, 4, 6, 64), (1, 3, 16, 128), (1, 2, 50, 128), (2, 2, 2, 256), (1, 1, 2, 128)])
def test_conv_fp32_stream_epilogue(S, engine, shape):
    """EVX_NN_EPI_RESID32: the FP32 stream in `pre` is updated in place (stream +=
    conv + bias, within FP32 accumulation of the FP64 oracle's conv) and `out`
    receives its BF16 copy; both engines (Z a multiple of 128: the pipelined
    kernel, whose epilogue stages the sums through shared memory; Y = 50 gives
    ragged y segments, X = 1 and Y = 2 wrap every neighbour onto the tile)."""
    import torch
    rng = np.random.default_rng(31 + engine + shape[2])
    x = bf16(rng.standard_normal(shape + (32,)))
    w = bf16(rng.standard_normal((27, 32, 32)) * 0.1)
    b = torch.from_numpy(rng.standard_normal(32).astype(np.float32))
    stream0 = rng.standard_normal(shape + (32,)).astype(np.float32)
    xd, wd, bd = x.cuda(), w.cuda(), b.cuda()
    h32 = torch.from_numpy(stream0).cuda()
    out = torch.empty(shape + (32,), dtype=torch.bfloat16, device="cuda")
    B, X, Y, Z = shape
    S.set_conv_engine(engine)
    try:
        S._ck(S.lib.evx_nn_conv3d(S._p(xd), S._p(wd), S._p(bd), S._p(out), S._p(h32), None,
                                  B, X, Y, Z, 32, 32, S.EPI_RESID32, S._stream()))
        S.check()
    finally:
        S.set_conv_engine(S.ENGINE_TCGEN05)
    ref = stream0.astype(np.float64) + N.conv(x.float().numpy().astype(np.float64),
                                              w.float().numpy().astype(np.float64), b.numpy().astype(np.float64))
    got32 = h32.cpu().numpy()
    assert rel(got32, ref) < 5e-6  # FP32 accumulation, no BF16 rounding of the stream
    assert rel(out.float().cpu().numpy(), ref) < 8e-3
    assert torch.equal(out.cpu(), torch.from_numpy(got32).to(torch.bfloat16))


@pytest.mark.parametrize("shape", [(2, 4, 6, 64), (1, 1, 2, 32), (1, 3, 5, 7), (2, 3, 4, 160)])
def test_fp32_stream_lift_and_projection(S, shape):
    """evx_nn_lift32 (unrounded field, FP32 sums and their BF16 copy) and
    evx_nn_project32 (reads the FP32 stream) against the FP64 oracle's conv.
    Z a multiple of 32 with Y even takes the lane-per-channel kernels (X = 1,
    Y = 2, Z = 32 wraps every neighbour onto the warp's own rows), other sizes
    the voxel-per-thread ones."""
    import torch
    rng = np.random.default_rng(12 + sum(shape))
    B, X, Y, Z = shape
    f = rng.uniform(-0.5, 0.5, shape).astype(np.float32)
    w0 = bf16(rng.standard_normal((27, 32, 16)) * 0.2)
    b0 = torch.from_numpy(rng.standard_normal(32).astype(np.float32))
    out = torch.empty(shape + (32,), dtype=torch.bfloat16, device="cuda")
    out32 = torch.empty(shape + (32,), dtype=torch.float32, device="cuda")
    fd, w0d, b0d = torch.from_numpy(f).cuda(), w0.cuda(), b0.cuda()
    S._ck(S.lib.evx_nn_lift32(S._p(fd), 1.0, S._p(w0d), 16, 32, S._p(b0d), S._p(out), S._p(out32),
                              B, X, Y, Z, S._stream()))
    xin = np.zeros(shape + (16,))
    xin[..., 0] = f
    ref = N.conv(xin, w0.float().numpy().astype(np.float64), b0.numpy().astype(np.float64))
    assert rel(out32.cpu().numpy(), ref) < 2e-6
    assert rel(out.float().cpu().numpy(), ref) < 8e-3
    h32 = rng.standard_normal(shape + (32,)).astype(np.float32)
    wp = bf16(rng.standard_normal((27, 16, 32)) * 0.1)
    bp = torch.from_numpy(rng.standard_normal(16).astype(np.float32))
    d = torch.empty(shape, dtype=torch.float32, device="cuda")
    h32d, wpd, bpd = torch.from_numpy(h32).cuda(), wp.cuda(), bp.cuda()
    S._ck(S.lib.evx_nn_project32(S._p(h32d), S._p(wpd), 32, 16, S._p(bpd), S._p(d), B, X, Y, Z, S._stream()))
    refp = N.conv(h32.astype(np.float64), wp.float().numpy().astype(np.float64), bp.numpy().astype(np.float64))[..., 0]
    assert rel(d.cpu().numpy(), refp) < 5e-6


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("shape", [(1, 3, 16, 128), (2, 4, 6, 64)])
def test_gelu_epilogue_without_pre(S, engine, shape):
    """EVX_NN_EPI_GELU with pre = NULL (inference) writes the same GELU output
    and nothing else."""
    import torch
    rng = np.random.default_rng(77 + engine + shape[3])
    x = bf16(rng.standard_normal(shape + (32,))).cuda()
    w = bf16(rng.standard_normal((27, 32, 32)) * 0.1).cuda()
    b = torch.from_numpy(rng.standard_normal(32).astype(np.float32)).cuda()
    B, X, Y, Z = shape
    outs = []
    S.set_conv_engine(engine)
    try:
        for keep in (True, False):
            out = torch.empty(shape + (32,), dtype=torch.bfloat16, device="cuda")
            pre = torch.zeros(shape + (32,), dtype=torch.bfloat16, device="cuda")
            S._ck(S.lib.evx_nn_conv3d(S._p(x), S._p(w), S._p(b), S._p(out), S._p(pre if keep else None), None,
                                      B, X, Y, Z, 32, 32, S.EPI_GELU, S._stream()))
            S.check()
            outs.append((out, pre))
    finally:
        S.set_conv_engine(S.ENGINE_TCGEN05)
    assert torch.equal(outs[0][0], outs[1][0])
    assert outs[0][1].abs().sum() > 0 and outs[1][1].abs().sum() == 0
