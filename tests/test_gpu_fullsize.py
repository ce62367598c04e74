"""Parity at the full sizes of the benchmarked workloads, in the launch configuration that
bench.py times (graph-replayed steps, default tuning), against the FP64 oracle on the same
seeded inputs (the oracle runs these sizes in seconds on the host cores)."""
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


def test_real_time_256cubed_fp64(orc):
    """256^3, h = 0.1, trap (0.5, 1, 1.5), g = 40, gdd = 25, dt = 5e-4, seeded Gaussian."""
    shape, h, nu, g, gdd, dt = (256, 256, 256), 0.1, (0.5, 1.0, 1.5), 40.0, 25.0, 5e-4
    psi0 = inputs.gaussian_psi(shape, h, noise=1e-3, seed=1)
    gpu = abi.Condensate(shape, h, dt, mode=abi.DGPE_REAL_TIME, nu=nu, g=g, gdd=gdd)
    gpu.set_psi(psi0)
    gpu.step(2)
    got = gpu.get_psi()
    o = gpu.observables()
    gpu.close()
    p = orc.make_params(shape, h, dt, orc.REAL_TIME, nu, g, gdd)
    want = orc.step(p, psi0, 2)
    assert rel(got, want) < 1e-10
    ow = orc.observables(p, want)
    # mu and E weight the psi difference by the discrete Laplacian (spectral radius
    # 4(1/hx^2 + 1/hy^2 + 1/hz^2) = 1200 at h = 0.1), so their bound is looser than psi's
    assert o["norm"] == pytest.approx(ow["norm"], rel=1e-11)
    for k in ("mu", "energy"):
        assert o[k] == pytest.approx(ow[k], rel=1e-9)


def test_imaginary_time_256cubed_fp64(orc):
    shape, h, nu, g, gdd, dt = (256, 256, 256), 0.1, (0.5, 1.0, 1.5), 50.0, 25.0, 0.004
    psi0 = inputs.gaussian_psi(shape, h, noise=1e-3, seed=1)
    gpu = abi.Condensate(shape, h, dt, mode=abi.DGPE_IMAG_TIME, nu=nu, g=g, gdd=gdd)
    gpu.set_psi(psi0)
    gpu.step(2)
    got = gpu.get_psi()
    gpu.close()
    want = orc.step(orc.make_params(shape, h, dt, orc.IMAG_TIME, nu, g, gdd), psi0, 2)
    assert rel(got, want) < 1e-10


def test_mixed_512x512x384(orc):
    """512x512x384, h = 0.05, trap (1, 1, 2), g = 100, gdd = 60, real time dt = 5e-4, one
    FP32-mixed step against the FP64 oracle (bound: FP32 rounding of psi and of the
    transforms, with margin), and the FP64 GPU path on the same input."""
    shape, h, nu, g, gdd, dt = (512, 512, 384), 0.05, (1.0, 1.0, 2.0), 100.0, 60.0, 5e-4
    psi0 = inputs.gaussian_psi(shape, h, noise=1e-3, seed=1).astype(np.complex64)
    gpu = abi.Condensate(shape, h, dt, mode=abi.DGPE_REAL_TIME, precision=abi.DGPE_MIXED, nu=nu, g=g, gdd=gdd)
    gpu.set_psi(psi0)
    gpu.step(1)
    got = gpu.get_psi().astype(np.complex128)
    gpu.close()
    want = orc.step(orc.make_params(shape, h, dt, orc.REAL_TIME, nu, g, gdd), psi0.astype(np.complex128), 1)
    err = rel(got, want)
    assert err < 2e-6, err
    del want
    g64 = abi.Condensate(shape, h, dt, mode=abi.DGPE_REAL_TIME, precision=abi.DGPE_FP64, nu=nu, g=g, gdd=gdd)
    g64.set_psi(psi0.astype(np.complex128))
    g64.step(1)
    ref64 = g64.get_psi()
    g64.close()
    assert rel(got, ref64) < 2e-6


def test_maximum_size_512cubed_fp64(orc):
    """Every axis at the largest supported length (512), FP64 real time, one step against
    the oracle; then double-float on the same input against the FP64 GPU result."""
    import torch
    shape, h, nu, g, gdd, dt = (512, 512, 512), 0.05, (1.0, 1.0, 2.0), 100.0, 60.0, 5e-4
    psi0 = inputs.gaussian_psi(shape, h, noise=1e-3, seed=2)
    gpu = abi.Condensate(shape, h, dt, mode=abi.DGPE_REAL_TIME, nu=nu, g=g, gdd=gdd)
    gpu.set_psi(psi0)
    gpu.step(1)
    got = gpu.get_psi(host=False)
    gpu.close()
    want = orc.step(orc.make_params(shape, h, dt, orc.REAL_TIME, nu, g, gdd), psi0, 1)
    assert rel(got.cpu().numpy(), want) < 1e-10
    del want
    dfc = abi.Condensate(shape, h, dt, mode=abi.DGPE_REAL_TIME, precision=abi.DGPE_DF64, nu=nu, g=g, gdd=gdd)
    dfc.set_psi(psi0)
    dfc.step(1)
    got_df = dfc.get_psi(host=False)
    dfc.close()
    assert float(torch.linalg.norm(got_df - got) / torch.linalg.norm(got)) < 1e-11


def test_adjoint_step_128cubed(orc):
    import torch
    shape, h, dt = (128, 128, 128), 0.2, 0.001
    gpu = abi.Condensate(shape, h, dt, mode=abi.DGPE_REAL_TIME, nu=(1.0, 1.0, 1.1), g=30.0, gdd=15.0)
    psi = inputs.gaussian_psi(shape, h, seed=4)
    w = inputs.random_psi(shape, seed=9)
    gbar = torch.from_numpy(w).cuda()
    gpu.adjoint_grads(reset=True)
    gpu.adjoint_step(torch.from_numpy(psi).cuda(), gbar)
    grads = gpu.adjoint_grads(reset=True)
    gpu.close()
    want, wgr = orc.adjoint_step(orc.make_params(shape, h, dt, orc.REAL_TIME, (1.0, 1.0, 1.1), 30.0, 15.0), psi, w)
    assert rel(gbar.cpu().numpy(), want) < 1e-11
    for q in range(3):
        assert grads[q] == pytest.approx(wgr[q], rel=1e-9)


@pytest.mark.parametrize("n", [32, 48, 64, 96, 128])
def test_batching_sizes_mixed(orc, n):
    """One member of each cube size of the batching workload (h = 12.8/N, imaginary time,
    FP32-mixed) after 10 steps, against the oracle."""
    h = 12.8 / n
    nu, g, gdd = (0.8, 1.4, 1.9), 45.0, 30.0
    psi0 = inputs.gaussian_psi((n, n, n), h, noise=1e-3, seed=n).astype(np.complex64)
    gpu = abi.Condensate((n, n, n), h, 0.001, mode=abi.DGPE_IMAG_TIME, precision=abi.DGPE_MIXED, nu=nu, g=g,
                         gdd=gdd)
    gpu.set_psi(psi0)
    gpu.step(10)
    got = gpu.get_psi().astype(np.complex128)
    gpu.close()
    want = orc.step(orc.make_params((n, n, n), h, 0.001, orc.IMAG_TIME, nu, g, gdd), psi0.astype(np.complex128), 10)
    assert rel(got, want) < 5e-6


def test_paper_grid_480x480x250_fp64(orc):
    """The grid of the paper's CUDA/MPI timings (Table 3): 480 x 480 x 250 (radix 2, 3, 5)."""
    shape, h, nu, g, gdd, dt = (480, 480, 250), 0.05, (1.0, 1.0, 1.5), 40.0, 20.0, 5e-4
    psi0 = inputs.gaussian_psi(shape, h, noise=1e-3, seed=2)
    gpu = abi.Condensate(shape, h, dt, mode=abi.DGPE_REAL_TIME, nu=nu, g=g, gdd=gdd)
    gpu.set_psi(psi0)
    gpu.step(1)
    got = gpu.get_psi()
    gpu.close()
    want = orc.step(orc.make_params(shape, h, dt, orc.REAL_TIME, nu, g, gdd), psi0, 1)
    assert rel(got, want) < 1e-10
