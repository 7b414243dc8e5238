"""The allocation-free step entry point (evx_ch_step_static).

Some callers cannot allocate device memory - their device memory belongs to
another runtime, or their footprint is fixed at start-up. For them the
library keeps every scratch buffer of the step in one static device array.
This checks, through the C-ABI, that two calls in a row give the same fields
as the regular grid path (evx_set_field / evx_ch_step / evx_get_field) to
the one-step parity tolerance, and that oversize grids are refused. The file
is named to be collected last.
"""
import numpy as np
import pytest

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


def grid_path(evx, c0, n, **p):
    import torch
    g = evx.Grid(c0.shape, **p)
    g.set_field(torch.from_numpy(c0).cuda())
    g.step(n)
    out = g.get_field().cpu().numpy()
    g.close()
    return out


def test_static_entry_point_matches_grid_path(evx):
    import torch
    cases = [((64, 64, 64), 0, 0.3, 5, dict(dt=0.1, M=1.0, kappa=1.0, h=1.0)),
             ((48, 40, 36), 7, 0.0, 3, dict(dt=0.05, M=0.7, kappa=1.6, h=0.9))]
    for shape, seed, offset, n, p in cases:  # two calls in a row, different shapes
        c0 = inputs.uniform_field(shape, seed=seed, offset=offset)
        cin = torch.from_numpy(c0).cuda()
        cout = torch.empty_like(cin)
        evx.ch_step_static(cin, cout, n, **p)
        torch.cuda.synchronize()
        ref = grid_path(evx, c0, n, **p)
        assert rel_l2(cout.cpu().numpy(), ref) <= 1e-5


def test_static_entry_point_in_place_allocates_nothing(evx):
    """d_c_out may equal d_c_in; the device's free memory is the same before and
    after two more calls (the first call of the process has already looked up the
    static array's address)."""
    import torch
    shape, n, p = (64, 64, 64), 4, dict(dt=0.1, M=1.0, kappa=1.0, h=1.0)
    c0 = inputs.uniform_field(shape, seed=11, offset=0.1)
    ref = grid_path(evx, c0, n, **p)
    buf = torch.from_numpy(c0).cuda()
    evx.ch_step_static(buf, buf, n, **p)  # in place
    torch.cuda.synchronize()
    assert rel_l2(buf.cpu().numpy(), ref) <= 1e-5
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        buf.copy_(torch.from_numpy(c0))
        evx.ch_step_static(buf, buf, n, **p)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    assert rel_l2(buf.cpu().numpy(), ref) <= 1e-5


def test_static_entry_point_rejects_oversize(evx):
    import torch
    c = torch.zeros((128, 64, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(evx.EvxError) as ei:
        evx.ch_step_static(c, c, 1)
    assert ei.value.status == evx.EVX_ERR_SIZE
