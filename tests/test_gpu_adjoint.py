"""GPU adjoint (differentiation workload) against the oracle's adjoint, and against central
finite differences of the GPU's own forward trajectory."""
import numpy as np
import pytest

from paper_1610_05329_gb300 import abi, inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1610_05329_gb300 import build
    build.build()
    abi.load()


@pytest.mark.parametrize("shape,h", [((8, 12, 16), 0.6), ((16, 18, 24), 0.45), ((32, 24, 36), 0.3)])
def test_adjoint_step_matches_oracle(orc, shape, h):
    import torch
    nu, g, gdd, dt = (1.0, 1.2, 0.9), 30.0, 18.0, 0.01
    gpu = abi.Condensate(shape, h, dt, mode=abi.DGPE_REAL_TIME, nu=nu, g=g, gdd=gdd)
    p = orc.make_params(shape, h, dt, orc.REAL_TIME, nu, g, gdd)
    psi = inputs.gaussian_psi(shape, h, seed=4)
    w = inputs.random_psi(shape, seed=9)
    psi_d = torch.from_numpy(psi).cuda()
    gbar = torch.from_numpy(w).cuda()
    gpu.adjoint_grads(reset=True)
    gpu.adjoint_step(psi_d, gbar)
    grads = gpu.adjoint_grads(reset=True)
    want, wgr = orc.adjoint_step(p, psi, w)
    assert rel(gbar.cpu().numpy(), want) < 1e-11
    for q in range(3):
        assert grads[q] == pytest.approx(wgr[q], rel=1e-9, abs=1e-13)
    gpu.close()


@pytest.mark.parametrize("nseg,spb", [(3, 4), (5, 3)])
def test_schedule_gradient_matches_oracle(orc, nseg, spb):
    shape, h, dt, g, gdd = (12, 16, 18), 0.5, 0.02, 30.0, 18.0
    nu_z = np.linspace(0.85, 1.2, nseg)
    psi0 = inputs.gaussian_psi(shape, h, seed=6, center=(0.2, -0.1, 0.3))
    gpu = abi.Condensate(shape, h, dt, mode=abi.DGPE_REAL_TIME, nu=(1.0, 1.2, 0.9), g=g, gdd=gdd)
    gpu.set_psi(psi0)
    loss, dnu, dg, dgdd = gpu.grad_z2(nu_z, spb)
    p = orc.make_params(shape, h, dt, orc.REAL_TIME, (1.0, 1.2, 0.9), g, gdd)
    wl, wdnu, wdg, wdgdd = orc.grad_z2(p, nu_z, spb, psi0)
    assert loss == pytest.approx(wl, rel=1e-11)
    assert rel(dnu, wdnu) < 1e-9
    assert dg == pytest.approx(wdg, rel=1e-9)
    assert dgdd == pytest.approx(wdgdd, rel=1e-9)
    # the context is back at the initial state
    assert rel(gpu.get_psi(), psi0) < 1e-15
    gpu.close()


def test_gpu_gradient_by_central_differences():
    """Central FD (h = 1e-6, FP64) of the GPU's own loss for g, gdd and two segments."""
    shape, hh, dt = (16, 16, 18), 0.45, 0.01
    nu_z = np.array([0.95, 1.1, 1.02, 0.9])
    spb = 5
    psi0 = inputs.gaussian_psi(shape, hh, seed=7, center=(0.0, 0.2, -0.3))

    def run(nu=nu_z, g=25.0, gdd=12.0):
        gpu = abi.Condensate(shape, hh, dt, mode=abi.DGPE_REAL_TIME, nu=(1.0, 1.1, 1.0), g=g, gdd=gdd)
        gpu.set_psi(psi0)
        out = gpu.grad_z2(nu, spb)
        gpu.close()
        return out

    loss, dnu, dg, dgdd = run()
    eps = 1e-6
    fd_g = (run(g=25.0 + eps)[0] - run(g=25.0 - eps)[0]) / (2 * eps)
    fd_gdd = (run(gdd=12.0 + eps)[0] - run(gdd=12.0 - eps)[0]) / (2 * eps)
    assert dg == pytest.approx(fd_g, rel=2e-6, abs=1e-10)
    assert dgdd == pytest.approx(fd_gdd, rel=2e-6, abs=1e-10)
    for s in (0, 2):
        up, dn = nu_z.copy(), nu_z.copy()
        up[s] += eps
        dn[s] -= eps
        fd = (run(nu=up)[0] - run(nu=dn)[0]) / (2 * eps)
        assert dnu[s] == pytest.approx(fd, rel=2e-6, abs=1e-10)


# (the second: short-line x and y sweeps; the third: the adjoint's compile-time z transforms)
@pytest.mark.parametrize("shape", [(24, 24, 24), (32, 48, 24), (16, 20, 128)])
def test_mixed_precision_gradient_vs_fp64(shape):
    h, dt = 0.4, 0.01
    nu_z = np.array([0.9, 1.1, 1.0])
    psi0 = inputs.gaussian_psi(shape, h, seed=8, center=(0.1, 0.0, 0.25))
    res = {}
    for prec in (abi.DGPE_FP64, abi.DGPE_MIXED):
        gpu = abi.Condensate(shape, h, dt, mode=abi.DGPE_REAL_TIME, precision=prec, nu=(1, 1, 1), g=30, gdd=15)
        gpu.set_psi(psi0.astype(np.complex128 if prec == abi.DGPE_FP64 else np.complex64))
        res[prec] = gpu.grad_z2(nu_z, 6)
        gpu.close()
    l64, d64, g64, gdd64 = res[abi.DGPE_FP64]
    l32, d32, g32, gdd32 = res[abi.DGPE_MIXED]
    assert l32 == pytest.approx(l64, rel=1e-5)
    assert rel(d32, d64) < 1e-3
    assert g32 == pytest.approx(g64, rel=1e-3, abs=1e-7)


def test_autograd_function():
    import torch
    shape, h, dt = (12, 12, 18), 0.5, 0.02
    psi0 = inputs.gaussian_psi(shape, h, seed=3, center=(0.0, 0.0, 0.2))
    gpu = abi.Condensate(shape, h, dt, mode=abi.DGPE_REAL_TIME, nu=(1, 1, 1), g=20, gdd=10)
    gpu.set_psi(psi0)
    nu = torch.tensor([1.0, 0.9, 1.1], dtype=torch.float64, requires_grad=True)
    g = torch.tensor(20.0, dtype=torch.float64, requires_grad=True)
    gdd = torch.tensor(10.0, dtype=torch.float64, requires_grad=True)
    loss = abi.trajectory_z2(gpu, nu, g, gdd, 4)
    (3.0 * loss).backward()
    l, dnu, dg, dgdd = gpu.grad_z2(np.array([1.0, 0.9, 1.1]), 4)
    assert float(loss.detach()) == pytest.approx(l, rel=1e-13)
    assert np.allclose(nu.grad.numpy(), 3.0 * dnu, rtol=1e-12)
    assert float(g.grad) == pytest.approx(3.0 * dg, rel=1e-12)
    assert float(gdd.grad) == pytest.approx(3.0 * dgdd, rel=1e-12)
    gpu.close()
