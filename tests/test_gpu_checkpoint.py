"""Checkpoint / resume and the host-side allocation-failure hook, through the
C-ABI.

* A run saved after 50 steps and resumed in a fresh grid gives, after 50 more,
  bit-for-bit the field of an uninterrupted 100-step run (each model; step
  graphs of 16 steps and single steps both occur on either side).
* evx_load refuses files of another size or model, corrupt and truncated
  files, and leaves the grid unchanged when it does.
* EVX_FAIL_ALLOC=k makes the k-th device allocation of a call fail without
  calling cudaMalloc: the call returns EVX_ERR_OOM, frees what it allocated and
  leaves the grid usable. No GPU fault is involved.
"""
import os

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


@pytest.mark.parametrize("model,shape", [("ch", (64, 64, 64)), ("ch", (48, 40, 36)), ("ac", (64, 128, 128)),
                                         ("vm", (32, 48, 40)), ("ch", (400, 64, 128))])
def test_resume_is_bitwise(evx, tmp_path, model, shape):
    import torch
    c0 = torch.from_numpy(inputs.uniform_field(shape, seed=12, offset=0.2)).cuda()
    p = dict(dt=0.1, M=0.9, kappa=1.2, h=1.0)
    ref = evx.Grid(shape, model=model, **p)
    ref.set_field(c0)
    ref.step(100)
    want = ref.get_field().cpu()
    E_want = ref.energy()
    ref.close()

    a = evx.Grid(shape, model=model, **p)
    a.set_field(c0)
    a.step(50)
    path = tmp_path / "run.evx"
    a.save(path)
    a.close()
    b = evx.Grid(shape, model=model, dt=0.5, M=2.0, kappa=3.0, h=1.0)  # parameters come from the file
    b.load(path)
    assert b.steps == 50
    assert (b.params.dt, b.params.M, b.params.kappa, b.params.h) == (0.1, 0.9, 1.2, 1.0)
    b.step(50)
    assert b.steps == 100
    got = b.get_field().cpu()
    E_got = b.energy()
    b.close()
    assert torch.equal(got, want)
    assert E_got == E_want


def test_load_refuses_mismatch_and_corruption(evx, tmp_path):
    import torch
    shape = (32, 32, 32)
    c0 = torch.from_numpy(inputs.uniform_field(shape, seed=3)).cuda()
    g = evx.Grid(shape)
    g.set_field(c0)
    g.step(3)
    path = tmp_path / "a.evx"
    g.save(path)
    before = g.get_field().cpu()

    other = evx.Grid((32, 32, 40))
    with pytest.raises(evx.EvxError) as ei:
        other.load(path)
    assert ei.value.status == evx.EVX_ERR_STATE
    other.close()
    ac = evx.Grid(shape, model="ac")
    with pytest.raises(evx.EvxError) as ei:
        ac.load(path)
    assert ei.value.status == evx.EVX_ERR_STATE
    ac.close()

    raw = bytearray(open(path, "rb").read())
    bad = tmp_path / "bad.evx"
    raw[-5] ^= 0x40  # one flipped payload bit
    open(bad, "wb").write(bytes(raw))
    for p in (bad, tmp_path / "missing.evx"):
        with pytest.raises(evx.EvxError) as ei:
            g.load(p)
        assert ei.value.status == evx.EVX_ERR_IO
    short = tmp_path / "short.evx"
    open(short, "wb").write(bytes(raw[: len(raw) // 2]))
    with pytest.raises(evx.EvxError) as ei:
        g.load(short)
    assert ei.value.status == evx.EVX_ERR_IO
    # the grid is untouched by the refused loads
    assert torch.equal(g.get_field().cpu(), before)
    assert g.steps == 3
    g.close()

    empty = evx.Grid(shape)
    with pytest.raises(evx.EvxError) as ei:
        empty.save(tmp_path / "none.evx")
    assert ei.value.status == evx.EVX_ERR_STATE
    empty.close()


@pytest.fixture
def fail_alloc():
    def set_k(k):
        if k is None:
            os.environ.pop("EVX_FAIL_ALLOC", None)
        else:
            os.environ["EVX_FAIL_ALLOC"] = str(k)
    yield set_k
    os.environ.pop("EVX_FAIL_ALLOC", None)


def test_injected_allocation_failure_in_create(evx, fail_alloc):
    import torch
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in (1, 2, 5):
        fail_alloc(k)
        with pytest.raises(evx.EvxError) as ei:
            evx.Grid((64, 64, 64))
        assert ei.value.status == evx.EVX_ERR_OOM
        assert "allocation %d of the call" % k in str(ei.value)
        assert torch.cuda.mem_get_info()[0] == free0  # what was allocated has been freed
    fail_alloc(None)
    g = evx.Grid((64, 64, 64))
    g.close()


def test_injected_allocation_failure_in_adjoint_and_model_switch(evx, fail_alloc):
    import torch
    shape = (32, 32, 32)
    c0 = torch.from_numpy(inputs.uniform_field(shape, seed=4)).cuda()
    g = evx.Grid(shape)
    g.set_field(c0)
    fp = g.footprint()
    for k in (1, 4):
        fail_alloc(k)
        with pytest.raises(evx.EvxError) as ei:
            g.adjoint(c0, 10, 5, torch.ones_like(c0))
        assert ei.value.status == evx.EVX_ERR_OOM
        assert g.footprint() == fp
    fail_alloc(1)
    with pytest.raises(evx.EvxError) as ei:
        g.set_model("vm")
    assert ei.value.status == evx.EVX_ERR_OOM
    assert g.model == "ch" and g.footprint() == fp
    fail_alloc(None)
    # the grid still works: an adjoint and a step run normally afterwards
    g0, gk, gm = g.adjoint(c0, 10, 5, torch.ones_like(c0))
    assert np.isfinite(gk) and np.isfinite(gm)
    g.set_field(c0)
    g.step(2)
    assert np.isfinite(g.energy()[0])
    g.close()
