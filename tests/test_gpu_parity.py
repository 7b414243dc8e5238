"""GPU parity of the CUDA Cahn-Hilliard step against the FP64 oracle.

Bars (from the method's stated accuracy targets): relative L2 <= 1e-5 after
one step and <= 1e-3 after 100 steps, FP32 bulk against the FP64 oracle, on
the same seeded FP32 inputs; the FP64 mean is carried exactly.
All calls go through the C-ABI (ctypes binding); nothing here runs on a CPU
fallback.
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


def gpu_run(evx, c0, nsteps, **params):
    import torch
    p = dict(dt=DT, M=M, kappa=KAPPA, h=H)
    p.update(params)
    g = evx.Grid(c0.shape, **p)
    g.set_field(torch.from_numpy(c0).cuda())
    g.step(nsteps)
    out = g.get_field().cpu().numpy()
    g.close()
    return out


# sizes that span several tiles, ragged column chunks and radix 3 / 5 stages
# (generic kernels), and power-of-two edges 64 .. 1024 (fast kernels, every
# threads-per-pencil variant, x, y and z)
SMALL = [(8, 8, 8), (16, 32, 64), (48, 40, 36), (24, 30, 50), (64, 64, 64)]
POW2 = [(64, 128, 256), (256, 512, 128), (512, 64, 1024), (1024, 256, 64), (128, 1024, 512)]
# lengths 400 = 20 x 20 along x and y and nz = 400 (M = 200 = 20 x 10) take the
# R1 = 20 fast kernels one axis at a time, next to power-of-two axes
MIXED = [(400, 64, 128), (64, 400, 128), (64, 128, 400)]


@pytest.mark.parametrize("shape", SMALL + [(400, 16, 20), (10, 1024, 12), (24, 400, 64), (16, 32, 400)])
def test_roundtrip(evx, shape):
    import torch
    c = inputs.uniform_field(shape, seed=3, offset=0.3)
    g = evx.Grid(shape)
    g.set_field(torch.from_numpy(c).cuda())
    back = g.get_field().cpu().numpy()
    mean = g.mean()
    g.close()
    assert np.abs(back - c).max() < 2e-6
    assert abs(mean - c.astype(np.float64).mean()) < 1e-15


@pytest.mark.parametrize("shape", SMALL + POW2 + MIXED + [(128, 128, 128)])
def test_one_step_vs_oracle(evx, shape):
    c0 = inputs.uniform_field(shape, seed=0)
    ref = O.ch_step(c0, DT, M, KAPPA, H, 1)
    got = gpu_run(evx, c0, 1)
    assert rel_l2(got, ref) <= 1e-5


@pytest.mark.parametrize("shape", [(64, 64, 64), (48, 40, 36), (128, 128, 128), (64, 128, 256)])
def test_100_steps_vs_oracle(evx, shape):
    c0 = inputs.uniform_field(shape, seed=0)
    ref = O.ch_step(c0, DT, M, KAPPA, H, 100, check_imag=False)
    got = gpu_run(evx, c0, 100)
    assert rel_l2(got, ref) <= 1e-3


@pytest.mark.parametrize("offset", [0.0, 0.3])
def test_parameters_and_offset(evx, offset):
    shape = (32, 40, 48)
    c0 = inputs.uniform_field(shape, seed=9, offset=offset, lo=-0.3, hi=0.3)
    ref = O.ch_step(c0, 0.05, 0.7, 1.6, 0.8, 5)
    got = gpu_run(evx, c0, 5, dt=0.05, M=0.7, kappa=1.6, h=0.8)
    assert rel_l2(got, ref) <= 1e-5


@pytest.mark.parametrize("n,plane", [(256, "xy"), (400, "xz")])
def test_100_steps_reduced_dimension(evx, n, plane):
    """A field constant along one axis evolves as the 2D problem; the oracle
    runs that 2D problem exactly and the whole 3D GPU field must match it."""
    shape2 = {"xy": (n, n, 1), "xz": (n, 1, n), "yz": (1, n, n)}[plane]
    c2 = inputs.uniform_field(shape2, seed=4)
    ref = O.ch_step(c2, DT, M, KAPPA, H, 100, check_imag=False)
    c3 = np.ascontiguousarray(np.broadcast_to(c2, (n, n, n)))
    got = gpu_run(evx, c3, 100)
    assert rel_l2(got, np.broadcast_to(ref, (n, n, n))) <= 1e-3


def test_one_step_400_cubed(evx):
    shape = (400, 400, 400)
    c0 = inputs.uniform_field(shape, seed=0)
    ref = O.ch_step(c0, DT, M, KAPPA, H, 1, check_imag=False)
    got = gpu_run(evx, c0, 1)
    assert rel_l2(got, ref) <= 1e-5


def test_mass_and_energy_trace(evx):
    import torch
    shape = (64, 64, 64)
    c0 = inputs.uniform_field(shape, seed=0)
    _, E_ref = O.ch_step(c0, DT, M, KAPPA, H, 100, energies=True, check_imag=False)
    g = evx.Grid(shape)
    g.set_field(torch.from_numpy(c0).cuda())
    mean0 = g.mean()
    Es = []
    for k in range(11):
        if k:
            g.step(10)
        E, mass = g.energy()
        Es.append(E)
        assert mass == mean0 * 64 ** 3  # FP64 mean carried exactly
    cN = g.get_field().cpu().numpy().astype(np.float64)
    g.close()
    Es = np.array(Es)
    assert np.all(np.diff(Es) < 0)
    assert np.abs(Es - E_ref[::10]).max() / np.abs(E_ref).max() < 1e-5
    # FP64 sum of the FP32 real field: drift bounded by FP32 rounding of the field
    l1 = np.abs(c0.astype(np.float64)).sum()
    assert abs(cN.sum() - c0.astype(np.float64).sum()) / l1 < 1e-6


def test_graph_and_profiled_paths_identical(evx):
    import torch
    shape = (48, 40, 36)
    c0 = torch.from_numpy(inputs.uniform_field(shape, seed=2)).cuda()
    outs = []
    for prof in (False, True):
        g = evx.Grid(shape)
        g.set_profiling(prof)
        g.set_field(c0)
        g.step(37)
        outs.append(g.get_field().cpu())
        if prof:
            ms, cnt = g.pass_times()
            assert cnt == [37, 37, 37, 37]
            assert all(m > 0 for m in ms)
        g.close()
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("shape", [(128, 256, 512), (400, 400, 400)])
def test_fast_and_generic_kernels_agree(evx, tmp_path, shape):
    """The fast kernels (R1 = 32 and R1 = 20 four-step splits) and the generic
    mixed-radix kernels (forced with EVX_GENERIC=1 in a child process) give the
    same field to FP32 rounding."""
    import subprocess
    import sys
    import torch
    c0 = inputs.uniform_field(shape, seed=8, offset=0.2)
    got = gpu_run(evx, c0, 10)
    script = (
        "import sys, numpy as np, torch\n"
        "sys.path.insert(0, %r)\n"
        "from paper_2507_21748_gb300 import evx, inputs\n"
        "c0 = inputs.uniform_field(%r, seed=8, offset=0.2)\n"
        "g = evx.Grid(%r, dt=0.1, M=1.0, kappa=1.0, h=1.0)\n"
        "g.set_field(torch.from_numpy(c0).cuda()); g.step(10)\n"
        "np.save(%r, g.get_field().cpu().numpy())\n"
    ) % (str(__import__("os").path.dirname(__import__("os").path.dirname(__file__))), shape, shape,
         str(tmp_path / "gen.npy"))
    env = dict(__import__("os").environ, EVX_GENERIC="1")
    subprocess.run([sys.executable, "-c", script], check=True, env=env)
    gen = np.load(tmp_path / "gen.npy")
    assert rel_l2(got, gen) <= 2e-6


@pytest.mark.parametrize("shape", [(32, 48, 40), (64, 128, 40), (24, 256, 64), (16, 400, 400)])
def test_host_io_matches_device_io(evx, shape):
    """Host copies (per y block of the spectral layout) equal the device path."""
    import torch
    c0 = inputs.uniform_field(shape, seed=5, offset=0.1)
    g = evx.Grid(shape)
    g.set_field_host(torch.from_numpy(c0))
    g.step(3)
    a = g.get_field_host().clone()
    b = g.get_field().cpu()
    g2 = evx.Grid(shape)
    g2.set_field(torch.from_numpy(c0).cuda())
    g2.step(3)
    c = g2.get_field().cpu()
    pageable = torch.empty(shape, dtype=torch.float32)  # not pinned: the staged copy path
    g.get_field_host(pageable)
    g.close()
    g2.close()
    assert torch.equal(a, b)
    assert torch.equal(a, c)
    assert torch.equal(pageable, b)


def test_nonfinite_detected(evx):
    import torch
    shape = (16, 16, 16)
    c0 = inputs.uniform_field(shape, seed=1)
    c0[3, 4, 5] = np.nan
    g = evx.Grid(shape)
    g.set_field(torch.from_numpy(c0).cuda())
    with pytest.raises(evx.EvxError) as ei:
        g.energy()
    assert ei.value.status == evx.EVX_ERR_NONFINITE
    g.close()


def test_state_errors(evx):
    g = evx.Grid((8, 8, 8))
    with pytest.raises(evx.EvxError) as ei:
        g.step(1)
    assert ei.value.status == evx.EVX_ERR_STATE
    with pytest.raises(evx.EvxError):
        g.energy()
    g.close()


def test_zero_mobility_identity_and_constant_fixed_point(evx):
    shape = (16, 24, 20)
    c0 = inputs.uniform_field(shape, seed=6, lo=-0.8, hi=0.8)
    got = gpu_run(evx, c0, 5, M=0.0)
    assert np.abs(got - c0).max() < 2e-6
    cc = np.full(shape, 0.37, dtype=np.float32)
    got = gpu_run(evx, cc, 5)
    assert np.abs(got - cc).max() < 1e-6


@pytest.mark.parametrize("n", [256, 400])
def test_1000_steps_statistics_and_footprint(evx, n):
    """The 256^3 and 400^3 configurations run for 1000 steps: parity is checked at
    1 and 100 steps elsewhere; here the FP64 mean is conserved exactly, the energy
    decays at every 100-step sample, the field stays bounded, and the grid holds
    two half-spectrum fields plus tables (no per-step allocation)."""
    import torch
    shape = (n, n, n)
    c0 = inputs.uniform_field(shape, seed=0)
    g = evx.Grid(shape)
    g.set_field(torch.from_numpy(c0).cuda())
    m0 = g.mean()
    E = [g.energy()[0]]
    free0 = None
    for _ in range(10):
        g.step(100)
        E.append(g.energy()[0])
        assert g.mean() == m0
        if free0 is None:  # after the first call has captured its step graphs
            free0 = torch.cuda.mem_get_info()[0]
    assert torch.cuda.mem_get_info()[0] == free0  # nothing allocated while stepping
    c = g.get_field()
    assert float(c.abs().max()) < 1.2
    Zp = ((n // 2 + 1) + 7) // 8 * 8
    field = n * n * Zp * 8
    assert g.footprint() <= 2 * field + 16 * 2 ** 20
    g.close()
    assert all(b <= a * (1 + 1e-9) for a, b in zip(E, E[1:]))
    assert E[-1] < 0.99 * E[0]
