"""GPU parity of the Allen-Cahn model (evx_set_model(EVX_MODEL_AC)) against
the FP64 oracle's ``ac_step``: the same four step passes with the Allen-Cahn
symbols and the FP64 mean moved by -dt L mean(c^3 - c) each step.

Bars, as for Cahn-Hilliard: relative L2 <= 1e-5 after one step and <= 1e-3
after 100 steps (FP32 bulk, FP64 oracle, the same seeded FP32 inputs). The
carried FP64 mean is checked against the oracle's mean: after one step within
1e-9 (its only error source is the FP32 rounding of the per-thread sums of
g(c) - g(cbar)); after many steps within the field's own bar (the mean is a
linear functional of the field, |mean(e)| <= rel_l2 * rms; the mean dynamics
near cbar = 0 amplify differences by about exp(L t), 2e4 over 100 steps), and
always within FP32 rounding of the mean of the field it belongs to.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_21748_gb300 import inputs

pytestmark = pytest.mark.gpu

DT, L, KAPPA, H = 0.1, 1.0, 1.0, 1.0


@pytest.fixture(scope="module")
def evx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_21748_gb300 import evx as E
    return E


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def ac_run(evx, c0, nsteps, **params):
    import torch
    p = dict(dt=DT, M=L, kappa=KAPPA, h=H)
    p.update(params)
    g = evx.Grid(c0.shape, model="ac", **p)
    g.set_field(torch.from_numpy(c0).cuda())
    g.step(nsteps)
    out = g.get_field().cpu().numpy()
    mean = g.mean()
    g.close()
    return out, mean


# fast power-of-two kernels, generic radix 2/3/5 kernels, ragged chunks
SHAPES = [(64, 64, 64), (48, 40, 36), (16, 32, 64), (24, 30, 50), (128, 64, 256)]


@pytest.mark.parametrize("shape", SHAPES)
def test_one_step_vs_oracle(evx, shape):
    c0 = inputs.uniform_field(shape, seed=11, offset=0.2)
    ref = O.ac_step(c0, DT, L, KAPPA, H, 1)
    got, mean = ac_run(evx, c0, 1)
    assert rel_l2(got, ref) <= 1e-5
    assert abs(mean - ref.mean()) <= 1e-9


@pytest.mark.parametrize("shape,offset", [((64, 64, 64), 0.0), ((48, 40, 36), 0.3), ((32, 64, 128), -0.2)])
def test_100_steps_vs_oracle(evx, shape, offset):
    c0 = inputs.uniform_field(shape, seed=12, offset=offset)
    ref = O.ac_step(c0, DT, L, KAPPA, H, 100, check_imag=False)
    got, mean = ac_run(evx, c0, 100)
    assert rel_l2(got, ref) <= 1e-3
    check_long_run_mean(got, ref, mean)


def rms(a):
    return float(np.sqrt(np.mean(np.asarray(a, np.float64) ** 2)))


def check_long_run_mean(got, ref, mean):
    assert abs(mean - ref.mean()) <= 1e-3 * rms(ref)
    assert abs(mean - np.asarray(got, np.float64).mean()) <= 1e-6 * rms(got)


def test_parameters(evx):
    shape = (40, 48, 64)
    c0 = inputs.uniform_field(shape, seed=13, offset=-0.1)
    ref = O.ac_step(c0, 0.05, 0.7, 1.6, 0.8, 5)
    got, mean = ac_run(evx, c0, 5, dt=0.05, M=0.7, kappa=1.6, h=0.8)
    assert rel_l2(got, ref) <= 1e-5
    assert abs(mean - ref.mean()) <= 1e-9


@pytest.mark.parametrize("n", [256])
def test_100_steps_reduced_dimension(evx, n):
    """A field constant along x evolves as the 2D problem; the oracle runs that
    problem exactly and the whole 3D GPU field (fast kernels) must match it."""
    c2 = inputs.uniform_field((1, n, n), seed=14, offset=0.1)
    ref = O.ac_step(c2, DT, L, KAPPA, H, 100, check_imag=False)
    c3 = np.ascontiguousarray(np.broadcast_to(c2, (n, n, n)))
    got, mean = ac_run(evx, c3, 100)
    assert rel_l2(got, np.broadcast_to(ref, (n, n, n))) <= 1e-3
    check_long_run_mean(got, np.broadcast_to(ref, (n, n, n)), mean)


def test_constant_field_mean_follows_the_scalar_recurrence(evx):
    # only the k = 0 mode: the device's FP64 mean update alone, exact to FP64 rounding
    shape = (64, 64, 64)
    c0 = np.full(shape, 0.37, dtype=np.float32)
    got, mean = ac_run(evx, c0, 25, dt=0.1, M=1.3, kappa=0.7)
    ref = float(np.float32(0.37))
    for _ in range(25):
        ref = ref - 0.1 * 1.3 * (ref ** 3 - ref)
    assert abs(mean - ref) <= 1e-14
    assert np.abs(got - ref).max() <= 1e-6  # FP32 field = FP32(mean)


def test_energy_decays_and_mean_moves(evx):
    import torch
    shape = (64, 64, 64)
    c0 = inputs.uniform_field(shape, seed=15, offset=0.1)
    g = evx.Grid(shape, model="ac", dt=DT, M=L, kappa=KAPPA, h=H)
    g.set_field(torch.from_numpy(c0).cuda())
    E = [g.energy()[0]]
    means = [g.mean()]
    for _ in range(20):
        g.step(2)
        E.append(g.energy()[0])
        means.append(g.mean())
    g.close()
    assert all(b <= a * (1 + 1e-6) for a, b in zip(E, E[1:]))
    assert E[-1] < E[0]
    assert means[-1] > means[0] + 0.01  # off-critical field drifts toward the +1 well


def test_graph_and_profiled_paths_identical(evx):
    import torch
    shape = (48, 40, 36)
    c0 = torch.from_numpy(inputs.uniform_field(shape, seed=16, offset=0.2)).cuda()
    outs = []
    for prof in (False, True):
        g = evx.Grid(shape, model="ac")
        g.set_profiling(prof)
        g.set_field(c0)
        g.step(37)
        outs.append((g.get_field().cpu(), g.mean()))
        g.close()
    assert torch.equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]


@pytest.mark.parametrize("shape", [(128, 256, 128), (400, 400, 400)])
def test_fast_and_generic_kernels_agree(evx, tmp_path, shape):
    import os
    import subprocess
    import sys
    c0 = inputs.uniform_field(shape, seed=17, offset=0.2)
    got, mean = ac_run(evx, c0, 10)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = (
        "import sys, numpy as np, torch\n"
        "sys.path.insert(0, %r)\n"
        "from paper_2507_21748_gb300 import evx, inputs\n"
        "c0 = inputs.uniform_field(%r, seed=17, offset=0.2)\n"
        "g = evx.Grid(%r, dt=0.1, M=1.0, kappa=1.0, h=1.0, model='ac')\n"
        "g.set_field(torch.from_numpy(c0).cuda()); g.step(10)\n"
        "np.save(%r, g.get_field().cpu().numpy()); np.save(%r, np.array([g.mean()]))\n"
    ) % (root, shape, shape, str(tmp_path / "gen.npy"), str(tmp_path / "mean.npy"))
    subprocess.run([sys.executable, "-c", script], check=True, env=dict(os.environ, EVX_GENERIC="1"))
    assert rel_l2(got, np.load(tmp_path / "gen.npy")) <= 2e-6
    # the fast path sums g(c) - g(cbar) in FP32 per thread and tile before FP64, the
    # generic one in FP64 per element: <= 1e-11 apart per step (one-step bars above)
    assert abs(mean - float(np.load(tmp_path / "mean.npy")[0])) <= 10 * 1e-11


def test_model_switching_and_guards(evx):
    import torch
    shape = (32, 32, 32)
    c0 = inputs.uniform_field(shape, seed=18, offset=0.2)
    g = evx.Grid(shape)
    assert g.model == "ch"
    g.set_field(torch.from_numpy(c0).cuda())
    g.step(3)  # CH
    g.set_model("ac")
    assert g.model == "ac"
    with pytest.raises(evx.EvxError):
        g._ck(evx.lib.evx_ch_step(g._h, 1))
    g.step(4)  # AC
    got = g.get_field().cpu().numpy()
    ref = O.ac_step(O.ch_step(c0, DT, 1.0, KAPPA, H, 3), DT, L, KAPPA, H, 4)
    assert rel_l2(got, ref) <= 1e-5
    dummy = torch.zeros(shape, dtype=torch.float32, device="cuda")
    with pytest.raises(evx.EvxError):
        g._ck(evx.lib.evx_ch_adjoint(g._h, evx.ctypes.c_void_p(dummy.data_ptr()), 2, 1,
                                     evx.ctypes.c_void_p(dummy.data_ptr()), evx.ctypes.c_void_p(dummy.data_ptr()),
                                     None, None))
    with pytest.raises(ValueError):
        g.set_model("gray-scott")
    g.set_model("ch")
    g.step(1)
    g.close()
