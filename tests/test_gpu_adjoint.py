"""GPU discrete adjoint (evx_ch_adjoint) against the FP64 oracle adjoint and
central finite differences, and the torch.autograd wrapper around it.

Loss (inverse problem of the method): L = 1/2 sum_x (c_N - c*)^2, c* the field
reached with other parameters.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_21748_gb300 import inputs

pytestmark = pytest.mark.gpu

DT, H = 0.1, 1.0


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


def forward(evx, c0, n, M, kappa):
    import torch
    g = evx.Grid(c0.shape, dt=DT, M=M, kappa=kappa, h=H)
    g.set_field(torch.from_numpy(c0).cuda())
    g.step(n)
    out = g.get_field().cpu().numpy().astype(np.float64)
    g.close()
    return out


def gpu_adjoint(evx, c0, n, ckpt, M, kappa, dLdcN):
    import torch
    g = evx.Grid(c0.shape, dt=DT, M=M, kappa=kappa, h=H)
    g0, gk, gm = g.adjoint(torch.from_numpy(c0).cuda(), n, ckpt,
                           torch.from_numpy(dLdcN.astype(np.float32)).cuda())
    g0 = g0.cpu().numpy().astype(np.float64)
    g.close()
    return g0, gk, gm


@pytest.mark.parametrize("shape,n,ckpt", [((24, 20, 16), 7, 3), ((32, 32, 32), 12, 5),
                                          ((64, 64, 64), 40, 20), ((128, 64, 256), 10, 4),
                                          ((400, 16, 24), 6, 3), ((1024, 8, 16), 5, 5)])
def test_adjoint_vs_oracle(evx, shape, n, ckpt):
    c0 = inputs.uniform_field(shape, seed=21, lo=-0.3, hi=0.3, offset=0.1)
    target = O.ch_step(c0, DT, 0.8, 1.5, H, n, check_imag=False)
    cN = O.ch_step(c0, DT, 1.0, 1.0, H, n, check_imag=False)
    dLdcN = (cN - target).astype(np.float32)
    ref0, refk, refm = O.ch_adjoint(c0, dLdcN.astype(np.float64), DT, 1.0, 1.0, H, n)
    g0, gk, gm = gpu_adjoint(evx, c0, n, ckpt, 1.0, 1.0, dLdcN)
    assert rel_l2(g0, ref0) <= 1e-4
    assert abs(gk - refk) <= 1e-4 * abs(refk)
    assert abs(gm - refm) <= 1e-4 * abs(refm)


def test_checkpoint_interval_does_not_change_result(evx):
    shape, n = (32, 24, 40), 13
    c0 = inputs.uniform_field(shape, seed=3, lo=-0.3, hi=0.3)
    rng = np.random.default_rng(0)
    dL = rng.standard_normal(shape).astype(np.float32)
    res = [gpu_adjoint(evx, c0, n, ck, 1.0, 1.0, dL) for ck in (1, 4, 13)]
    for g0, gk, gm in res[1:]:
        assert np.array_equal(g0, res[0][0])
        assert gk == res[0][1] and gm == res[0][2]


def test_inverse_problem_128_central_differences(evx):
    """128^3, target from 200 steps with kappa = 1.5, M = 0.8, loss from kappa = M = 1,
    checkpoint every 20 steps; dL/dkappa, dL/dM and dL/dc0 . d against central
    differences (step 1e-3) of the GPU forward solve."""
    shape, n = (128, 128, 128), 200
    c0 = inputs.uniform_field(shape, seed=0)
    target = forward(evx, c0, n, 0.8, 1.5)

    def loss(c0_, M, kappa):
        cN = forward(evx, c0_, n, M, kappa)
        return 0.5 * float(np.sum((cN - target) ** 2))

    cN = forward(evx, c0, n, 1.0, 1.0)
    g0, gk, gm = gpu_adjoint(evx, c0, n, 20, 1.0, 1.0, (cN - target).astype(np.float32))
    e = 1e-3
    fd_k = (loss(c0, 1.0, 1.0 + e) - loss(c0, 1.0, 1.0 - e)) / (2 * e)
    fd_m = (loss(c0, 1.0 + e, 1.0) - loss(c0, 1.0 - e, 1.0)) / (2 * e)
    assert abs(fd_k - gk) <= 2e-3 * abs(gk), (fd_k, gk)
    assert abs(fd_m - gm) <= 2e-3 * abs(gm), (fd_m, gm)
    rng = np.random.default_rng(1)
    d = rng.standard_normal(shape)
    d *= 0.01 / np.abs(d).max()
    # step of 1e-3 along d: perturbations of the FP32 input stay resolvable
    cp = (c0 + 0.1 * d).astype(np.float32)
    cm = (c0 - 0.1 * d).astype(np.float32)
    fd_c = (loss(cp, 1.0, 1.0) - loss(cm, 1.0, 1.0)) / 2.0
    an_c = float(np.sum(g0 * (cp.astype(np.float64) - cm.astype(np.float64)))) / 2.0
    assert abs(fd_c - an_c) <= 1e-2 * abs(an_c), (fd_c, an_c)


def test_autograd_function(evx):
    import torch
    shape, n = (32, 32, 32), 10
    c0 = inputs.uniform_field(shape, seed=5, lo=-0.3, hi=0.3)
    target = torch.from_numpy(O.ch_step(c0, DT, 0.8, 1.5, H, n).astype(np.float32)).cuda()
    g = evx.Grid(shape, dt=DT, M=1.0, kappa=1.0, h=H)
    x = torch.from_numpy(c0).cuda().requires_grad_(True)
    kappa = torch.tensor(1.0, dtype=torch.float64, device="cuda", requires_grad=True)
    M = torch.tensor(1.0, dtype=torch.float64, device="cuda", requires_grad=True)
    cN = evx.ch_solve(x, kappa, M, g, n, ckpt_every=4)
    loss = 0.5 * ((cN.double() - target.double()) ** 2).sum()
    loss.backward()
    ref0, refk, refm = O.ch_adjoint(c0, (O.ch_step(c0, DT, 1.0, 1.0, H, n) - target.cpu().numpy()),
                                    DT, 1.0, 1.0, H, n)
    assert rel_l2(x.grad.cpu().numpy(), ref0) <= 1e-4
    assert abs(float(kappa.grad) - refk) <= 1e-4 * abs(refk)
    assert abs(float(M.grad) - refm) <= 1e-4 * abs(refm)
    g.close()
