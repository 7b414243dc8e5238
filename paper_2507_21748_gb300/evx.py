"""Thin ctypes binding of libevx.so (C-ABI in include/evx.h).

Argument marshalling only: every step of the solver runs in the CUDA
library. PyTorch supplies device memory and streams. Importing this module
loads the library and raises if it has not been built (there is no CPU
fallback).
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# EVX_LIB selects another build of the same library (the bounds-checked
# libevx_bounds.so of the debug tests); default: the normal build
LIB_PATH = os.environ.get("EVX_LIB") or os.path.join(_HERE, "_lib", "libevx.so")

(EVX_OK, EVX_ERR_ARG, EVX_ERR_SIZE, EVX_ERR_OOM, EVX_ERR_CUDA, EVX_ERR_NONFINITE, EVX_ERR_STATE,
 EVX_ERR_IO) = range(8)
STATUS_NAMES = ["EVX_OK", "EVX_ERR_ARG", "EVX_ERR_SIZE", "EVX_ERR_OOM", "EVX_ERR_CUDA",
                "EVX_ERR_NONFINITE", "EVX_ERR_STATE", "EVX_ERR_IO"]

# every entry point declared in include/evx.h
EXPORTS = [
    "evx_grid_create", "evx_grid_destroy", "evx_set_params", "evx_get_params", "evx_set_stream", "evx_set_field",
    "evx_set_field_host", "evx_get_field", "evx_get_field_host", "evx_ch_step", "evx_ch_block", "evx_energy",
    "evx_mean", "evx_ch_adjoint", "evx_footprint", "evx_set_profiling", "evx_pass_times",
    "evx_pass_bytes", "evx_ch_step_static", "evx_set_model", "evx_get_model", "evx_step", "evx_step_count",
    "evx_save", "evx_load", "evx_debug_bounds", "evx_last_error",
]
MODELS = {"ch": 0, "ac": 1, "vm": 2}  # evx_model: Cahn-Hilliard, Allen-Cahn, variable-mobility CH


class EvxError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s: %s" % (name, msg))


class Params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("M", ctypes.c_double), ("kappa", ctypes.c_double),
                ("h", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libevx.so not built (%s); run __graft_entry__.build() first" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, dp, fp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p
    i, st = ctypes.c_int, ctypes.c_int
    sig = {
        "evx_grid_create": ([i, i, i, Params, vp, ctypes.POINTER(vp)], st),
        "evx_grid_destroy": ([vp], st),
        "evx_set_params": ([vp, Params], st),
        "evx_get_params": ([vp, ctypes.POINTER(Params)], st),
        "evx_set_stream": ([vp, vp], st),
        "evx_set_field": ([vp, fp], st),
        "evx_set_field_host": ([vp, fp], st),
        "evx_get_field": ([vp, fp], st),
        "evx_get_field_host": ([vp, fp], st),
        "evx_ch_step": ([vp, i], st),
        "evx_ch_block": ([vp, i], st),
        "evx_energy": ([vp, dp, dp], st),
        "evx_mean": ([vp, dp], st),
        "evx_ch_adjoint": ([vp, fp, i, i, fp, fp, dp, dp], st),
        "evx_footprint": ([vp, ctypes.POINTER(ctypes.c_size_t)], st),
        "evx_set_profiling": ([vp, i], st),
        "evx_pass_times": ([vp, dp, ctypes.POINTER(ctypes.c_longlong), i], st),
        "evx_pass_bytes": ([vp, i, dp], st),
        "evx_ch_step_static": ([fp, fp, i, i, i, Params, i, vp], st),
        "evx_set_model": ([vp, i], st),
        "evx_get_model": ([vp], ctypes.c_int),
        "evx_step": ([vp, i], st),
        "evx_step_count": ([vp, ctypes.POINTER(ctypes.c_longlong)], st),
        "evx_save": ([vp, ctypes.c_char_p], st),
        "evx_load": ([vp, ctypes.c_char_p], st),
        "evx_debug_bounds": ([ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], st),
        "evx_last_error": ([vp], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check_field(t, shape):
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != torch.float32:
        raise TypeError("expected a float32 CUDA tensor")
    if tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError("expected a contiguous tensor of shape %s" % (tuple(shape),))


class Grid:
    """A periodic nx*ny*nz grid owned by libevx, stepping the Cahn-Hilliard model
    (``model="ch"``, default), the Allen-Cahn model (``model="ac"``, M is then
    the kinetic coefficient L) or Cahn-Hilliard with variable mobility
    M max(1 - c^2, 0) and a finite-difference right-hand side (``model="vm"``)."""

    def __init__(self, shape, dt=0.1, M=1.0, kappa=1.0, h=1.0, stream=None, model="ch"):
        self.shape = tuple(int(s) for s in shape)
        self.params = Params(dt, M, kappa, h)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h_ = ctypes.c_void_p()
        s = lib.evx_grid_create(*self.shape, self.params, _stream_handle(self.stream), ctypes.byref(h_))
        if s != EVX_OK:
            raise EvxError(s, lib.evx_last_error(None).decode())
        self._h = h_
        if model != "ch":
            self.set_model(model)

    # -- helpers
    def _ck(self, s):
        if s != EVX_OK:
            raise EvxError(s, lib.evx_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib.evx_grid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- API
    def set_params(self, dt=None, M=None, kappa=None, h=None):
        p = self.params
        self.params = Params(p.dt if dt is None else dt, p.M if M is None else M,
                             p.kappa if kappa is None else kappa, p.h if h is None else h)
        self._ck(lib.evx_set_params(self._h, self.params))

    def set_field(self, c):
        _check_field(c, self.shape)
        self._ck(lib.evx_set_field(self._h, ctypes.c_void_p(c.data_ptr())))

    def set_field_host(self, c_host):
        assert c_host.dtype == torch.float32 and c_host.is_contiguous() and c_host.device.type == "cpu"
        assert tuple(c_host.shape) == self.shape
        self._ck(lib.evx_set_field_host(self._h, ctypes.c_void_p(c_host.data_ptr())))

    def get_field(self, out=None):
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        _check_field(out, self.shape)
        self._ck(lib.evx_get_field(self._h, ctypes.c_void_p(out.data_ptr())))
        return out

    def get_field_host(self, out=None):
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32).pin_memory()
        assert out.dtype == torch.float32 and out.is_contiguous() and tuple(out.shape) == self.shape
        self._ck(lib.evx_get_field_host(self._h, ctypes.c_void_p(out.data_ptr())))
        return out

    def set_model(self, model):
        if model not in MODELS:
            raise ValueError("model must be one of %s" % sorted(MODELS))
        self._ck(lib.evx_set_model(self._h, MODELS[model]))

    @property
    def model(self):
        m = lib.evx_get_model(self._h)
        return {v: k for k, v in MODELS.items()}[m]

    def step(self, n=1):
        self._ck(lib.evx_step(self._h, int(n)))

    @property
    def steps(self):
        n = ctypes.c_longlong()
        self._ck(lib.evx_step_count(self._h, ctypes.byref(n)))
        return n.value

    def save(self, path):
        """Write a checkpoint (state, FP64 mean, parameters, step count) to path."""
        self._ck(lib.evx_save(self._h, os.fsencode(str(path))))

    def load(self, path):
        """Resume from a checkpoint written by save() for a grid of this size and model."""
        self._ck(lib.evx_load(self._h, os.fsencode(str(path))))
        p = Params()  # the checkpoint carries its parameters
        self._ck(lib.evx_get_params(self._h, ctypes.byref(p)))
        self.params = p

    def block(self, n=10):
        """One block of n steps: linear part exact, nonlinear remainder frozen (evx_ch_block)."""
        self._ck(lib.evx_ch_block(self._h, int(n)))

    def energy(self):
        E = ctypes.c_double()
        m = ctypes.c_double()
        self._ck(lib.evx_energy(self._h, ctypes.byref(E), ctypes.byref(m)))
        return E.value, m.value

    def mean(self):
        c = ctypes.c_double()
        self._ck(lib.evx_mean(self._h, ctypes.byref(c)))
        return c.value

    def footprint(self):
        b = ctypes.c_size_t()
        self._ck(lib.evx_footprint(self._h, ctypes.byref(b)))
        return b.value

    def set_profiling(self, on):
        self._ck(lib.evx_set_profiling(self._h, 1 if on else 0))

    def pass_times(self, reset=False):
        ms = (ctypes.c_double * 4)()
        cnt = (ctypes.c_longlong * 4)()
        self._ck(lib.evx_pass_times(self._h, ms, cnt, 1 if reset else 0))
        return list(ms), list(cnt)

    def pass_bytes(self, k):
        b = ctypes.c_double()
        self._ck(lib.evx_pass_bytes(self._h, int(k), ctypes.byref(b)))
        return b.value

    def adjoint(self, c0, n_steps, ckpt_every, dLdcN, dLdc0=None):
        """Gradients of a loss of c_N: returns (dL/dc0, dL/dkappa, dL/dM)."""
        _check_field(c0, self.shape)
        _check_field(dLdcN, self.shape)
        if dLdc0 is None:
            dLdc0 = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        gk = ctypes.c_double()
        gm = ctypes.c_double()
        self._ck(lib.evx_ch_adjoint(self._h, ctypes.c_void_p(c0.data_ptr()), int(n_steps),
                                    int(ckpt_every), ctypes.c_void_p(dLdcN.data_ptr()),
                                    ctypes.c_void_p(dLdc0.data_ptr()), ctypes.byref(gk),
                                    ctypes.byref(gm)))
        return dLdc0, gk.value, gm.value


def debug_bounds():
    """(enabled, line): whether this is the bounds-checked build, and the source line
    of the first out-of-bounds access the checked kernels skipped since the last
    call (0 if none). Synchronises the device."""
    en, line = ctypes.c_int(), ctypes.c_int()
    s = lib.evx_debug_bounds(ctypes.byref(en), ctypes.byref(line))
    if s != EVX_OK:
        raise EvxError(s, lib.evx_last_error(None).decode())
    return en.value, line.value


def ch_step_static(c_in, c_out, n_steps, dt=0.1, M=1.0, kappa=1.0, h=1.0, stream=None):
    """Allocation-free step (evx_ch_step_static): c_out <- n_steps steps from c_in.

    Scratch lives in the library's static device array (grids up to 64^3);
    calls share it, so they must not overlap on the GPU."""
    shape = tuple(c_in.shape)
    _check_field(c_in, shape)
    _check_field(c_out, shape)
    s = lib.evx_ch_step_static(ctypes.c_void_p(c_in.data_ptr()), ctypes.c_void_p(c_out.data_ptr()),
                               *shape, Params(dt, M, kappa, h), int(n_steps), _stream_handle(stream))
    if s != EVX_OK:
        raise EvxError(s, lib.evx_last_error(None).decode())
    return c_out


class CHSolve(torch.autograd.Function):
    """c_N = n_steps semi-implicit CH steps from c0, differentiable in c0, kappa, M.

    Forward and backward both run in libevx (the backward is the hand-written
    discrete adjoint with checkpoint-every-k recomputation)."""

    @staticmethod
    def forward(ctx, c0, kappa, M, grid, n_steps, ckpt_every):
        grid.set_params(kappa=float(kappa), M=float(M))
        c0c = c0.detach().contiguous()
        grid.set_field(c0c)
        grid.step(n_steps)
        cN = grid.get_field()
        ctx.grid = grid
        ctx.n_steps = n_steps
        ctx.ckpt_every = ckpt_every
        ctx.kappa = float(kappa)
        ctx.M = float(M)
        ctx.param_like = (kappa, M)
        ctx.save_for_backward(c0c)
        return cN

    @staticmethod
    def backward(ctx, grad_out):
        (c0,) = ctx.saved_tensors
        grid = ctx.grid
        grid.set_params(kappa=ctx.kappa, M=ctx.M)
        g0, gk, gm = grid.adjoint(c0, ctx.n_steps, ctx.ckpt_every, grad_out.contiguous().float())

        def like(v, ref):
            if isinstance(ref, torch.Tensor):
                return torch.tensor(v, dtype=ref.dtype, device=ref.device).reshape(ref.shape)
            return None

        kappa, M = ctx.param_like
        return g0, like(gk, kappa), like(gm, M), None, None, None


def ch_solve(c0, kappa, M, grid, n_steps, ckpt_every=20):
    """Differentiable solve; kappa and M may be 0-d tensors with requires_grad."""
    return CHSolve.apply(c0, kappa, M, grid, n_steps, ckpt_every)
