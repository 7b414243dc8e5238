"""GPU parity of the variable-mobility Cahn-Hilliard model
(evx_set_model(EVX_MODEL_VM)) against the FP64 oracle's ``vm_step``: FD
right-hand side div(M(c) grad mu) in real space, spectral preconditioner
dt / (1 + dt M kappa |k|^4), real FP32 state.

Bars as for the constant-mobility model: relative L2 <= 1e-5 after one step and
<= 1e-3 after 100 steps on the same seeded FP32 inputs. Mass: the FD divergence
sums to zero and the update's k = 0 mode is dropped, so the FP64 mean of the
FP32 field moves only by the rounding of adding FP32 increments (about
1e-7 of an increment per voxel, unbiased): <= 1e-8 relative after 100 steps.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_21748_gb300 import inputs

pytestmark = pytest.mark.gpu

DT, M, KAPPA, H = 0.1, 1.0, 1.0, 1.0


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


def vm_run(evx, c0, nsteps, **params):
    import torch
    p = dict(dt=DT, M=M, kappa=KAPPA, h=H)
    p.update(params)
    g = evx.Grid(c0.shape, model="vm", **p)
    g.set_field(torch.from_numpy(c0).cuda())
    g.step(nsteps)
    out = g.get_field().cpu().numpy()
    mean = g.mean()
    E, mass = g.energy()
    g.close()
    return out, mean, E


SHAPES = [(64, 64, 64), (48, 40, 36), (16, 32, 64), (24, 30, 50), (128, 64, 256)]


@pytest.mark.parametrize("shape", SHAPES)
def test_one_step_vs_oracle(evx, shape):
    c0 = inputs.uniform_field(shape, seed=21, offset=0.2)
    ref = O.vm_step(c0, DT, M, KAPPA, H, 1)
    got, mean, E = vm_run(evx, c0, 1)
    assert rel_l2(got, ref) <= 1e-5
    # the increment itself, relative to its own size
    inc = ref - c0.astype(np.float64)
    assert rel_l2(got - c0, inc) <= 1e-4
    assert abs(E - O.vm_energy(ref, KAPPA, H)) <= 1e-5 * abs(O.vm_energy(ref, KAPPA, H))


@pytest.mark.parametrize("shape,offset", [((64, 64, 64), 0.0), ((48, 40, 36), 0.3)])
def test_100_steps_vs_oracle(evx, shape, offset):
    c0 = inputs.uniform_field(shape, seed=22, offset=offset)
    ref = O.vm_step(c0, DT, M, KAPPA, H, 100)
    got, mean, E = vm_run(evx, c0, 100)
    assert rel_l2(got, ref) <= 1e-3
    m0 = float(np.mean(c0.astype(np.float64)))
    assert abs(mean - m0) <= 1e-8 * max(abs(m0), float(np.mean(np.abs(c0))))


def test_parameters(evx):
    shape = (40, 48, 64)
    c0 = inputs.uniform_field(shape, seed=23, offset=-0.1)
    ref = O.vm_step(c0, 0.05, 0.7, 1.6, 0.8, 5)
    got, _, _ = vm_run(evx, c0, 5, dt=0.05, M=0.7, kappa=1.6, h=0.8)
    assert rel_l2(got, ref) <= 1e-5


def test_energy_decays(evx):
    import torch
    shape = (64, 64, 64)
    c0 = inputs.uniform_field(shape, seed=24, offset=0.1)
    g = evx.Grid(shape, model="vm")
    g.set_field(torch.from_numpy(c0).cuda())
    E = [g.energy()[0]]
    for _ in range(15):
        g.step(4)
        E.append(g.energy()[0])
    g.close()
    assert all(b <= a * (1 + 1e-6) for a, b in zip(E, E[1:]))
    assert E[-1] < E[0]


def test_graph_and_profiled_paths_identical(evx):
    import torch
    shape = (48, 40, 36)
    c0 = torch.from_numpy(inputs.uniform_field(shape, seed=25, offset=0.2)).cuda()
    outs = []
    for prof in (False, True):
        g = evx.Grid(shape, model="vm")
        g.set_profiling(prof)
        g.set_field(c0)
        g.step(21)
        outs.append(g.get_field().cpu())
        if prof:
            ms, cnt = g.pass_times()
            assert cnt == [21, 21, 21, 21]
        g.close()
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("shape", [(128, 256, 128), (400, 400, 400)])
def test_fast_and_generic_kernels_agree(evx, tmp_path, shape):
    import os
    import subprocess
    import sys
    c0 = inputs.uniform_field(shape, seed=26, offset=0.2)
    got, _, _ = vm_run(evx, c0, 10)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = (
        "import sys, numpy as np, torch\n"
        "sys.path.insert(0, %r)\n"
        "from paper_2507_21748_gb300 import evx, inputs\n"
        "c0 = inputs.uniform_field(%r, seed=26, offset=0.2)\n"
        "g = evx.Grid(%r, dt=0.1, M=1.0, kappa=1.0, h=1.0, model='vm')\n"
        "g.set_field(torch.from_numpy(c0).cuda()); g.step(10)\n"
        "np.save(%r, g.get_field().cpu().numpy())\n"
    ) % (root, shape, shape, str(tmp_path / "gen.npy"))
    subprocess.run([sys.executable, "-c", script], check=True, env=dict(os.environ, EVX_GENERIC="1"))
    assert rel_l2(got, np.load(tmp_path / "gen.npy")) <= 2e-6


def test_host_io_and_model_switching(evx):
    import torch
    shape = (32, 40, 48)
    c0 = inputs.uniform_field(shape, seed=27, offset=0.1)
    g = evx.Grid(shape)
    g.set_field(torch.from_numpy(c0).cuda())
    g.set_model("vm")
    with pytest.raises(evx.EvxError):  # the CH field does not carry over
        g.step(1)
    host = torch.from_numpy(c0).pin_memory()
    g.set_field_host(host)
    g.step(3)
    out = g.get_field_host().numpy()
    assert rel_l2(out, O.vm_step(c0, DT, M, KAPPA, H, 3)) <= 1e-5
    g.set_model("ch")
    with pytest.raises(evx.EvxError):
        g.step(1)
    g.set_field(torch.from_numpy(c0).cuda())
    g.step(1)
    assert rel_l2(g.get_field().cpu().numpy(), O.ch_step(c0, DT, M, KAPPA, H, 1)) <= 1e-5
    g.close()
