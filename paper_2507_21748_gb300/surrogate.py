"""Learned surrogate of the semi-implicit Cahn-Hilliard step (binding, training and guarded rollout).

A 3D residual CNN advances the field by a block of solver steps (C-ABI in
include/evx_nn.h). Every forward, backward and optimiser step runs in
libevx's kernels; PyTorch only provides device buffers. The plain solver
generates the training pairs, serves as fallback when the surrogate's mass
drift or energy increase exceeds a threshold, and measures its error against the solver.
"""
import ctypes
import time

import numpy as np
import torch

from . import evx, inputs

lib = evx.lib
NN_EXPORTS = ["evx_nn_conv3d", "evx_nn_conv3d_wgrad", "evx_nn_bias_grad", "evx_nn_flip_weights",
              "evx_nn_field_to_act", "evx_nn_zero_mean_add", "evx_nn_mse", "evx_nn_adam",
              "evx_nn_f32_to_bf16", "evx_nn_set_conv_engine", "evx_nn_conv_engine", "evx_nn_check",
              "evx_nn_lift", "evx_nn_project", "evx_nn_abs_sum", "evx_nn_zero_mean_add_scaled",
              "evx_nn_nl_scale", "evx_nn_lift32", "evx_nn_project32", "evx_nn_last_error"]
EPI_PLAIN, EPI_GELU, EPI_RESID, EPI_GELU_BWD, EPI_FIELD, EPI_RESID32 = range(6)
ENGINE_TCGEN05, ENGINE_MMA_SYNC = 0, 1


def _setup():
    vp, i, ll, f, st = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_float, ctypes.c_int
    sig = {
        "evx_nn_conv3d": [vp, vp, vp, vp, vp, vp, i, i, i, i, i, i, i, vp],
        "evx_nn_conv3d_wgrad": [vp, vp, vp, vp, ctypes.c_size_t, i, i, i, i, i, i, vp],
        "evx_nn_bias_grad": [vp, ll, i, vp, i, vp, vp],
        "evx_nn_flip_weights": [vp, i, i, vp, vp],
        "evx_nn_field_to_act": [vp, ll, i, f, vp, vp],
        "evx_nn_zero_mean_add": [vp, vp, i, ll, vp, i, vp, vp],
        "evx_nn_mse": [vp, vp, ll, f, vp, vp, i, vp, vp],
        "evx_nn_abs_sum": [vp, ll, vp, i, vp, vp],
        "evx_nn_zero_mean_add_scaled": [vp, vp, vp, i, ll, vp, i, vp, vp],
        "evx_nn_nl_scale": [vp, i, ll, vp, i, vp, vp],
        "evx_nn_adam": [vp, vp, vp, vp, i, f, f, f, f, i, vp, vp],
        "evx_nn_f32_to_bf16": [vp, i, vp, vp],
        "evx_nn_set_conv_engine": [i],
        "evx_nn_lift": [vp, f, vp, i, i, vp, vp, i, i, i, i, vp],
        "evx_nn_project": [vp, vp, i, i, vp, vp, i, i, i, i, vp],
        "evx_nn_lift32": [vp, f, vp, i, i, vp, vp, vp, i, i, i, i, vp],
        "evx_nn_project32": [vp, vp, i, i, vp, vp, i, i, i, i, vp],
        "evx_nn_conv_engine": [],
        "evx_nn_check": [],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = st
    lib.evx_nn_last_error.argtypes = []
    lib.evx_nn_last_error.restype = ctypes.c_char_p


_setup()


def _p(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _ck(s):
    if s != evx.EVX_OK:
        raise evx.EvxError(s, lib.evx_nn_last_error().decode())


def set_conv_engine(engine):
    """ENGINE_TCGEN05 (default) or ENGINE_MMA_SYNC for the 32 -> 32 convolutions."""
    _ck(lib.evx_nn_set_conv_engine(engine))


def conv_engine():
    return lib.evx_nn_conv_engine()


def check():
    """Synchronize and raise if a tensor-core pipeline wait ran past its bound."""
    _ck(lib.evx_nn_check())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Net:
    """lift 1->W, nblocks x [conv W->W, GELU, conv W->W] + skip, projection W->1.

    Parameters are FP32 masters with BF16 copies (and flipped BF16 copies for
    the data gradients); activations BF16 channels-last for `batch` fields
    of `shape`."""

    CIN = 16  # the input field is padded to 16 channels (channel 0 = c)
    CPROJ = 16  # the projection writes 16 channels, channel 0 is used

    def __init__(self, shape, batch, width=32, nblocks=4, seed=0, train=True, proj_gain=0.01, f32_stream=True):
        assert width == 32
        self.shape, self.batch, self.W, self.nb = tuple(shape), int(batch), width, nblocks
        # f32_stream: the residual stream h is kept in FP32 (the field enters the lift
        # unrounded, each block adds its output to the FP32 stream, the projection reads
        # it); the convolutions still take BF16 operands (a BF16 copy of the stream)
        self.f32 = bool(f32_stream)
        self.training = train
        self.V = int(np.prod(self.shape))
        self.nvox = self.V * self.batch
        dev = "cuda"
        rng = np.random.default_rng(seed)

        def w(co, ci, fan_in, gain):
            return (rng.standard_normal((27, co, ci)) * gain * np.sqrt(2.0 / fan_in)).astype(np.float32)

        W = self.W
        init = [("W0", w(W, self.CIN, 27, 1.0)), ("b0", np.zeros(W, np.float32))]
        for k in range(nblocks):
            init += [("W1_%d" % k, w(W, W, 27 * W, 1.0)), ("b1_%d" % k, np.zeros(W, np.float32)),
                     ("W2_%d" % k, w(W, W, 27 * W, 0.1)), ("b2_%d" % k, np.zeros(W, np.float32))]
        wp = w(self.CPROJ, W, 27 * W, proj_gain)
        wp[:, 1:, :] = 0.0  # only channel 0 of the projection reaches the output
        init += [("Wp", wp), ("bp", np.zeros(self.CPROJ, np.float32))]
        w0 = init[0][1]
        w0[:, :, 1:] = 0.0  # input channels 1.. are padding
        self.names = [n for n, _ in init]
        self.p = {n: torch.from_numpy(a).to(dev) for n, a in init}
        self.g = {n: torch.zeros_like(t) for n, t in self.p.items()}
        self.m = {n: torch.zeros_like(t) for n, t in self.p.items()}
        self.v = {n: torch.zeros_like(t) for n, t in self.p.items()}
        self.wbf = {n: torch.empty(t.shape, dtype=torch.bfloat16, device=dev)
                    for n, t in self.p.items() if n.startswith("W")}
        self.wflip = {n: torch.empty((27, t.shape[2], t.shape[1]), dtype=torch.bfloat16, device=dev)
                      for n, t in self.p.items() if n.startswith("W") and n != "W0"}
        self.step_count = 0
        self._refresh_bf16()
        # output scale of the base-corrected form (evx_nn_nl_scale), per sample
        self.scale = torch.zeros(self.batch, dtype=torch.float64, device=dev)
        self._scaled = False
        bf = torch.bfloat16
        nv = self.nvox
        # the padded lift input: for the lift's weight gradient, or for the tensor-core lift when W != 32
        self.a_in = torch.empty((nv, self.CIN), dtype=bf, device=dev) if (train or W != 32) else None
        if not train:
            # inference: the residual stream is updated in place; one GELU input and output
            # (the GELU pre-activations are not kept)
            h, a = (torch.empty((nv, W), dtype=bf, device=dev) for _ in range(2))
            self.h, self.u, self.a = [h] * (nblocks + 1), [None] * nblocks, [a] * nblocks
            self.h32 = torch.empty((nv, W), dtype=torch.float32, device=dev) if self.f32 else None
            self.d = torch.empty(nv, dtype=torch.float32, device=dev)
            self.pred = torch.empty(nv, dtype=torch.float32, device=dev)
            sms = torch.cuda.get_device_properties(0).multi_processor_count
            self.nparts = 2 * sms
            self.dpart = torch.empty(self.nparts * max(W, self.batch), dtype=torch.float64, device=dev)
            self.spart = torch.empty(3 * self.nparts * self.batch, dtype=torch.float64, device=dev)
            return
        self.h = [torch.empty((nv, W), dtype=bf, device=dev) for _ in range(nblocks + 1)]
        self.h32 = torch.empty((nv, W), dtype=torch.float32, device=dev) if self.f32 else None
        self.u = [torch.empty((nv, W), dtype=bf, device=dev) for _ in range(nblocks)]
        self.a = [torch.empty((nv, W), dtype=bf, device=dev) for _ in range(nblocks)]
        self.d = torch.empty(nv, dtype=torch.float32, device=dev)
        self.pred = torch.empty(nv, dtype=torch.float32, device=dev)
        self.gpred = torch.empty(nv, dtype=torch.float32, device=dev)
        self.gact = torch.empty((nv, self.CPROJ), dtype=bf, device=dev)
        self.dh = torch.empty((nv, W), dtype=bf, device=dev)
        self.du = torch.empty((nv, W), dtype=bf, device=dev)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        self.partial_floats = 2 * sms * 27 * W * W
        self.wpart = torch.empty(self.partial_floats, dtype=torch.float32, device=dev)
        self.nparts = 2 * sms
        self.dpart = torch.empty(self.nparts * max(W, self.batch), dtype=torch.float64, device=dev)
        self.spart = torch.empty(3 * self.nparts * self.batch, dtype=torch.float64, device=dev)
        self.dsum = torch.zeros(1, dtype=torch.float64, device=dev)

    # ---------------------------------------------------------- parameters
    def _refresh_bf16(self):
        s = _stream()
        for n, t in self.wbf.items():
            _ck(lib.evx_nn_f32_to_bf16(_p(self.p[n]), self.p[n].numel(), _p(t), s))
        for n, t in self.wflip.items():
            co, ci = self.p[n].shape[1], self.p[n].shape[2]
            _ck(lib.evx_nn_flip_weights(_p(self.wbf[n]), co, ci, _p(t), s))

    def load_params(self, other):
        """Take the parameters of another Net (e.g. trained at another size)."""
        for n in self.names:
            self.p[n].copy_(other.p[n])
        self._refresh_bf16()

    def params_numpy(self):
        """Parameters as the GPU uses them (BF16-rounded weights, FP32 biases), FP64."""
        out = {}
        for n, t in self.p.items():
            if n in self.wbf:
                out[n] = self.wbf[n].float().cpu().numpy().astype(np.float64)
            else:
                out[n] = t.cpu().numpy().astype(np.float64)
        return {"W0": out["W0"], "b0": out["b0"], "Wp": out["Wp"], "bp": out["bp"],
                "blocks": [(out["W1_%d" % k], out["b1_%d" % k], out["W2_%d" % k], out["b2_%d" % k])
                           for k in range(self.nb)]}

    # --------------------------------------------------------------- layers
    def _conv(self, inp, wname, bias, out, cin, cout, epi, pre=None, res=None, flipped=False):
        w = self.wflip[wname] if flipped else self.wbf[wname]
        X, Y, Z = self.shape
        _ck(lib.evx_nn_conv3d(_p(inp), _p(w), _p(bias), _p(out), _p(pre), _p(res), self.batch, X, Y, Z,
                              cin, cout, epi, _stream()))

    def _wgrad(self, dy, x, gname, cin, cout):
        X, Y, Z = self.shape
        _ck(lib.evx_nn_conv3d_wgrad(_p(dy), _p(x), _p(self.g[gname]), _p(self.wpart), self.partial_floats,
                                    self.batch, X, Y, Z, cin, cout, _stream()))

    def _bgrad(self, dy, gname, c):
        _ck(lib.evx_nn_bias_grad(_p(dy), self.nvox, c, _p(self.dpart), self.nparts, _p(self.g[gname]),
                                 _stream()))

    # -------------------------------------------------------------- forward
    def forward(self, c, base=None):
        """c: float32 CUDA tensor (batch, X, Y, Z) -> base + zero-mean correction,
        with base = c (the network predicts the whole block's increment) or the
        block propagator's prediction of the same block (the network predicts its
        error; see block_base)."""
        assert c.is_contiguous() and c.numel() == self.nvox and c.dtype == torch.float32
        if base is not None:
            assert base.is_contiguous() and base.shape == c.shape and base.dtype == torch.float32
        self._c = c
        s = _stream()
        W = self.W
        X, Y, Z = self.shape
        if self.training:  # the padded input is kept for the lift's weight gradient
            _ck(lib.evx_nn_field_to_act(_p(c), self.nvox, self.CIN, 1.0, _p(self.a_in), s))
        if W == 32 and self.f32:  # direct sum, FP32 stream and its BF16 copy
            _ck(lib.evx_nn_lift32(_p(c), 1.0, _p(self.wbf["W0"]), self.CIN, W, _p(self.p["b0"]), _p(self.h[0]),
                                  _p(self.h32), self.batch, X, Y, Z, s))
        elif W == 32:  # direct sum: only input channel 0 is nonzero
            _ck(lib.evx_nn_lift(_p(c), 1.0, _p(self.wbf["W0"]), self.CIN, W, _p(self.p["b0"]), _p(self.h[0]),
                                self.batch, X, Y, Z, s))
        else:
            if not self.training:
                _ck(lib.evx_nn_field_to_act(_p(c), self.nvox, self.CIN, 1.0, _p(self.a_in), s))
            self._conv(self.a_in, "W0", self.p["b0"], self.h[0], self.CIN, W, EPI_PLAIN)
        for k in range(self.nb):
            # the pre-activation is kept for the backward pass only
            self._conv(self.h[k], "W1_%d" % k, self.p["b1_%d" % k], self.a[k], W, W, EPI_GELU,
                       pre=self.u[k] if self.training else None)
            if self.f32:  # h32 += conv2(a); BF16 copy of the new stream into h[k + 1]
                self._conv(self.a[k], "W2_%d" % k, self.p["b2_%d" % k], self.h[k + 1], W, W, EPI_RESID32,
                           pre=self.h32)
            else:
                self._conv(self.a[k], "W2_%d" % k, self.p["b2_%d" % k], self.h[k + 1], W, W, EPI_RESID,
                           res=self.h[k])
        if W == 32 and self.f32:
            _ck(lib.evx_nn_project32(_p(self.h32), _p(self.wbf["Wp"]), W, self.CPROJ, _p(self.p["bp"]),
                                     _p(self.d), self.batch, X, Y, Z, s))
        elif W == 32:  # direct sum: only output channel 0 is used
            _ck(lib.evx_nn_project(_p(self.h[self.nb]), _p(self.wbf["Wp"]), W, self.CPROJ, _p(self.p["bp"]),
                                   _p(self.d), self.batch, X, Y, Z, s))
        else:
            self._conv(self.h[self.nb], "Wp", self.p["bp"], self.d, W, self.CPROJ, EPI_FIELD)
        self._scaled = base is not None
        if base is None:  # c + zero-mean correction
            _ck(lib.evx_nn_zero_mean_add(_p(c), _p(self.d), self.batch, self.V, _p(self.dpart), self.nparts,
                                         _p(self.pred), s))
        else:  # base + scale * zero-mean correction, scale = the nonlinearity's relative strength
            _ck(lib.evx_nn_nl_scale(_p(c), self.batch, self.V, _p(self.spart), self.nparts, _p(self.scale), s))
            _ck(lib.evx_nn_zero_mean_add_scaled(_p(base), _p(self.d), _p(self.scale), self.batch, self.V,
                                                _p(self.dpart), self.nparts, _p(self.pred), s))
        return self.pred.view(c.shape)

    # ------------------------------------------------------------- backward
    def loss(self, target):
        """Mean squared error of the last forward vs target (FP64 sum on the GPU)."""
        _ck(lib.evx_nn_mse(_p(self.pred), _p(target), self.nvox, 0.0, None, _p(self.dpart), self.nparts,
                           _p(self.dsum), _stream()))
        return float(self.dsum.item()) / self.nvox

    def backward(self, target):
        """Gradients of L = mean((pred - target)^2) into self.g; returns L."""
        assert self.training, "inference-only Net"
        s = _stream()
        W = self.W
        _ck(lib.evx_nn_mse(_p(self.pred), _p(target), self.nvox, 2.0 / self.nvox, _p(self.gpred),
                           _p(self.dpart), self.nparts, _p(self.dsum), s))
        # transpose of the (scaled) zero-mean projection is the projection itself
        if self._scaled:
            _ck(lib.evx_nn_zero_mean_add_scaled(None, _p(self.gpred), _p(self.scale), self.batch, self.V,
                                                _p(self.dpart), self.nparts, _p(self.gpred), s))
        else:
            _ck(lib.evx_nn_zero_mean_add(None, _p(self.gpred), self.batch, self.V, _p(self.dpart), self.nparts,
                                         _p(self.gpred), s))
        _ck(lib.evx_nn_field_to_act(_p(self.gpred), self.nvox, self.CPROJ, 1.0, _p(self.gact), s))
        self._wgrad(self.gact, self.h[self.nb], "Wp", W, self.CPROJ)
        self._bgrad(self.gact, "bp", self.CPROJ)
        self._conv(self.gact, "Wp", None, self.dh, self.CPROJ, W, EPI_PLAIN, flipped=True)
        for k in range(self.nb - 1, -1, -1):
            self._wgrad(self.dh, self.a[k], "W2_%d" % k, W, W)
            self._bgrad(self.dh, "b2_%d" % k, W)
            self._conv(self.dh, "W2_%d" % k, None, self.du, W, W, EPI_GELU_BWD, pre=self.u[k], flipped=True)
            self._wgrad(self.du, self.h[k], "W1_%d" % k, W, W)
            self._bgrad(self.du, "b1_%d" % k, W)
            self._conv(self.du, "W1_%d" % k, None, self.dh, W, W, EPI_RESID, res=self.dh, flipped=True)
        self._wgrad(self.dh, self.a_in, "W0", self.CIN, W)
        self._bgrad(self.dh, "b0", W)
        return float(self.dsum.item()) / self.nvox

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        s = _stream()
        for n in self.names:
            _ck(lib.evx_nn_adam(_p(self.p[n]), _p(self.g[n]), _p(self.m[n]), _p(self.v[n]), self.p[n].numel(),
                                lr, b1, b2, eps, self.step_count, None, s))
        self._refresh_bf16()


# ------------------------------------------------------------ base propagator
def block_base(grid, c, out, block=10):
    """The block propagator's prediction of c after `block` steps (evx_ch_block:
    the scheme's linear part exact over the block, its nonlinear remainder
    N = d^2 (3 cbar + d) frozen at the block's start; one step's cost). grid: an
    evx.Grid of c's shape and the scheme's parameters; c, out: (X, Y, Z) float32."""
    grid.set_field(c)
    grid.block(block)
    grid.get_field(out)


# ----------------------------------------------------------------- training
class TrajectoryPool:
    """B solver trajectories at `shape`, advanced `block` steps per draw; each
    starts from c0 = mean(seed) + U(-0.05, 0.05) and is restarted with the next
    seed after `horizon` steps (seeds cycle through first_seed .. last_seed).
    With base=True each draw also returns the block propagator's prediction of
    the block (block_base)."""

    def __init__(self, shape, batch, block=10, horizon=300, seeds=range(256), dt=0.1, M=1.0, kappa=1.0,
                 base=False):
        self.shape, self.batch, self.block, self.horizon = tuple(shape), batch, block, horizon
        self.seeds = list(seeds)
        self.next_seed = 0
        self.grids = [evx.Grid(shape, dt=dt, M=M, kappa=kappa) for _ in range(batch)]
        self.bgrid = evx.Grid(shape, dt=dt, M=M, kappa=kappa) if base else None
        self.age = [0] * batch
        self.cur = torch.empty((batch,) + self.shape, dtype=torch.float32, device="cuda")
        self.nxt = torch.empty_like(self.cur)
        self.bas = torch.empty_like(self.cur) if base else None
        for i in range(batch):
            self._restart(i)

    def _restart(self, i):
        seed = self.seeds[self.next_seed % len(self.seeds)]
        self.next_seed += 1
        c0 = inputs.uniform_field(self.shape, seed=seed, offset=inputs.trajectory_mean(seed))
        self.grids[i].set_field(torch.from_numpy(c0).cuda())
        self.age[i] = 0

    def draw(self):
        """(c_n, c_{n+block}) for every trajectory of the pool, and the block
        propagator's c_{n+block} when the pool was made with base=True."""
        for i, g in enumerate(self.grids):
            if self.age[i] >= self.horizon:
                self._restart(i)
            g.get_field(self.cur[i])
            if self.bgrid is not None:
                block_base(self.bgrid, self.cur[i], self.bas[i], self.block)
            g.step(self.block)
            g.get_field(self.nxt[i])
            self.age[i] += self.block
        return (self.cur, self.nxt) if self.bgrid is None else (self.cur, self.nxt, self.bas)

    def close(self):
        for g in self.grids:
            g.close()
        if self.bgrid is not None:
            self.bgrid.close()


def train(net, pool, iters, lr=2e-3, lr_final=2e-4, log_every=50, log=None):
    """Adam with a geometric learning-rate decay; returns the loss history."""
    hist = []
    for it in range(iters):
        batch = pool.draw()
        x, y = batch[0], batch[1]
        net.forward(x.contiguous(), batch[2].contiguous() if len(batch) > 2 else None)
        L = net.backward(y.contiguous())
        frac = it / max(iters - 1, 1)
        net.adam(lr * (lr_final / lr) ** frac)
        hist.append(L)
        if log and (it % log_every == 0 or it == iters - 1):
            log("iter %5d loss %.4e" % (it, L))
    return hist


# -------------------------------------------------------- guarded rollout
def rollout(net, c0, nblocks, block=10, dt=0.1, M=1.0, kappa=1.0, mass_tol=1e-6, energy_tol=1e-7, base=False):
    """Advance c0 (batch, X, Y, Z) by nblocks x block steps with the surrogate;
    a sample whose predicted block drifts in mass beyond mass_tol (relative
    to its L1 norm) or raises the energy beyond energy_tol (relative) is
    recomputed by the plain solver for that block. With base=True the network
    corrects the block propagator's prediction (block_base). Returns (fields, stats)."""
    shape = tuple(c0.shape[1:])
    B = c0.shape[0]
    referee = evx.Grid(shape, dt=dt, M=M, kappa=kappa)
    c = c0.clone()
    bas = torch.empty_like(c) if base else None
    nparts = 2 * torch.cuda.get_device_properties(0).multi_processor_count
    l1parts = torch.empty(nparts, dtype=torch.float64, device="cuda")
    l1sum = torch.empty(1, dtype=torch.float64, device="cuda")

    def l1(x):  # FP64 sum of |x| in the library
        _ck(lib.evx_nn_abs_sum(_p(x), x.numel(), _p(l1parts), nparts, _p(l1sum), _stream()))
        return float(l1sum.item())

    fallbacks = 0
    t_net = t_guard = t_fb = t_base = 0.0
    E_prev = [None] * B  # refereed energy and mass of each sample's current field
    for _ in range(nblocks):
        torch.cuda.synchronize()
        tb = time.perf_counter()
        if base:
            for i in range(B):
                block_base(referee, c[i], bas[i], block)
            torch.cuda.synchronize()
        t0 = time.perf_counter()
        t_base += t0 - tb
        pred = (net.forward(c.contiguous(), bas) if base else net.forward(c.contiguous())).clone()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        t_net += t1 - t0
        for i in range(B):
            if E_prev[i] is None:
                referee.set_field(c[i])
                E_prev[i] = referee.energy()
            E0, m0 = E_prev[i]
            l1n = l1(c[i])
            referee.set_field(pred[i])
            E1, m1 = referee.energy()
            ok = abs(m1 - m0) <= mass_tol * l1n and E1 <= E0 * (1 + energy_tol) + 1e-300
            E_prev[i] = (E1, m1)
            t2 = time.perf_counter()
            if not ok:
                referee.set_field(c[i])
                referee.step(block)
                referee.get_field(pred[i])
                E_prev[i] = None  # checked afresh next block
                fallbacks += 1
                torch.cuda.synchronize()
                t_fb += time.perf_counter() - t2
        t_guard += time.perf_counter() - t1
        c = pred
    referee.close()
    return c, {"fallbacks": fallbacks, "blocks": nblocks * B, "t_net_s": t_net, "t_guard_s": t_guard - t_fb,
               "t_fallback_s": t_fb, "t_base_s": t_base}


def base_rollout(c0, nblocks, block=10, dt=0.1, M=1.0, kappa=1.0):
    """The block propagator alone (no network, no guard): the method without the
    learned correction."""
    shape = tuple(c0.shape[1:])
    g = evx.Grid(shape, dt=dt, M=M, kappa=kappa)
    out = torch.empty_like(c0)
    for i in range(c0.shape[0]):
        g.set_field(c0[i].contiguous())
        for _ in range(nblocks):
            g.block(block)
        g.get_field(out[i])
    g.close()
    return out


def solver_run(c0, nsteps, dt=0.1, M=1.0, kappa=1.0):
    """Plain-solver reference for a batch of fields."""
    shape = tuple(c0.shape[1:])
    g = evx.Grid(shape, dt=dt, M=M, kappa=kappa)
    out = torch.empty_like(c0)
    for i in range(c0.shape[0]):
        g.set_field(c0[i].contiguous())
        g.step(nsteps)
        g.get_field(out[i])
    g.close()
    return out
