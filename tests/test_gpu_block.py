"""The block propagator (evx_ch_block: the scheme's linear part exact over a
block of n steps, its nonlinear remainder N = d^2 (3 cbar + d) frozen at the
block's start) against the FP64 oracle's ch_block_step, through the C-ABI, on
fast and mixed-radix sizes; n = 1 is one step of the scheme."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_21748_gb300 import inputs

pytestmark = pytest.mark.gpu


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


def gpu_block(evx, c0, n, nblocks=1, **p):
    import torch
    g = evx.Grid(c0.shape, **p)
    g.set_field(torch.from_numpy(c0).cuda())
    m0 = g.mean()
    for _ in range(nblocks):
        g.block(n)
    out = g.get_field().cpu().numpy()
    assert g.mean() == m0 and g.steps == n * nblocks
    g.close()
    return out


@pytest.mark.parametrize("shape", [(64, 64, 64), (128, 128, 128), (48, 40, 36), (400, 64, 128), (64, 128, 400)])
@pytest.mark.parametrize("offset", [0.0, 0.3])
def test_block_vs_oracle(evx, shape, offset):
    c0 = inputs.uniform_field(shape, seed=2, offset=offset, lo=-0.3, hi=0.3)
    p = dict(dt=0.1, M=0.9, kappa=1.1, h=1.0)
    ref = O.ch_block_step(c0, p["dt"], p["M"], p["kappa"], p["h"], 10)
    got = gpu_block(evx, c0, 10, **p)
    assert rel_l2(got, ref) <= 1e-5


def test_block_of_one_step_is_a_step(evx):
    import torch
    shape = (64, 64, 128)
    c0 = inputs.uniform_field(shape, seed=4, offset=0.1, lo=-0.5, hi=0.5)
    one = gpu_block(evx, c0, 1)
    g = evx.Grid(shape)
    g.set_field(torch.from_numpy(c0).cuda())
    g.step(1)
    stepped = g.get_field().cpu().numpy()
    g.close()
    assert rel_l2(one, stepped) <= 1e-6
    assert rel_l2(one, O.ch_step(c0, 0.1, 1.0, 1.0, 1.0, 1)) <= 1e-5


def test_block_refuses_other_models_and_bad_counts(evx):
    g = evx.Grid((16, 16, 16), model="ac")
    import torch
    g.set_field(torch.zeros((16, 16, 16), device="cuda"))
    with pytest.raises(evx.EvxError) as ei:
        g.block(10)
    assert ei.value.status == evx.EVX_ERR_STATE
    g.set_model("ch")
    with pytest.raises(evx.EvxError) as ei:
        g.block(0)
    assert ei.value.status == evx.EVX_ERR_ARG
    g.close()
