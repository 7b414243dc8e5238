"""The bounds-checked debug build (libevx_bounds.so, -DEVX_BOUNDS_CHECK) on
small and odd shapes: every global load and store of the mixed-radix,
adjoint, reduction and variable-mobility kernels tests its index against the
buffer; an access outside it is skipped and its source line recorded (no
trap). Runs every entry point that reaches those kernels in a child process
that loads the checked build (EVX_LIB), once with the mixed-radix kernels
forced everywhere (EVX_GENERIC=1) and once with the default dispatch, and
requires no recorded violation and finite results."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
sys.path.insert(0, %r)
import numpy as np, torch
from paper_2507_21748_gb300 import evx, inputs
en, line = evx.debug_bounds()
assert en == 1, "not the bounds-checked build"
shapes = [(8, 8, 8), (16, 32, 64), (48, 40, 36), (24, 30, 50), (10, 12, 18), (400, 16, 20), (64, 64, 128)]
for shape in shapes:
    c0 = torch.from_numpy(inputs.uniform_field(shape, seed=1, offset=0.1, lo=-0.4, hi=0.4)).cuda()
    for model in ("ch", "ac", "vm"):
        g = evx.Grid(shape, model=model)
        g.set_field(c0)
        g.step(3)
        E, m = g.energy()
        out = g.get_field()
        assert np.isfinite(E) and bool(torch.isfinite(out).all())
        if model == "ch":
            g.block(4)
            d0, gk, gm = g.adjoint(c0, 3, 2, torch.ones_like(c0))
            assert bool(torch.isfinite(d0).all()) and np.isfinite(gk) and np.isfinite(gm)
            host = g.get_field_host()
        g.close()
    if shape[0] * shape[1] * shape[2] <= 64 ** 3:
        o = torch.empty_like(c0)
        evx.ch_step_static(c0, o, 2)
print("BOUNDS", evx.debug_bounds()[1])
''' % ROOT


@pytest.fixture(scope="module")
def bounds_lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_21748_gb300.build import build_lib
    return build_lib(debug_bounds=True)


@pytest.mark.parametrize("generic", ["1", "0"])
def test_no_out_of_bounds_access(bounds_lib, generic):
    env = dict(os.environ, EVX_LIB=bounds_lib, EVX_GENERIC=generic)
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("BOUNDS")]
    assert lines and lines[-1] == "BOUNDS 0", r.stdout[-2000:]
