"""The double-float precision (DGPE_DF64: every value a pair of FP32 numbers, about 48
significant bits, all arithmetic on the FP32 pipe) against the FP64 oracle on the same
seeded inputs.  Bars: a pair carries ~2^-48 = 3.6e-15 relative precision, so sub-steps are
held to 1e-11 and multi-step runs to the FP64 path's 1e-10; the boundary (complex128 in
and out) loses only the bits below 2^-48."""
import numpy as np
import pytest

from paper_1610_05329_gb300 import abi, inputs

pytestmark = pytest.mark.gpu

DF_SUB_TOL = 1e-11
DF_STEP_TOL = 1e-10


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1610_05329_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    abi.load()


def make(orc, shape, h, dt, mode, nu=(1.0, 1.1, 0.9), g=25.0, gdd=15.0, **kw):
    gpu = abi.Condensate(shape, h, dt, mode=mode, precision=abi.DGPE_DF64, nu=nu, g=g, gdd=gdd, **kw)
    p = orc.make_params(shape, h, dt, orc.IMAG_TIME if mode == abi.DGPE_IMAG_TIME else orc.REAL_TIME, nu, g, gdd,
                        **kw)
    return gpu, p


def state(shape, h, seed=3):
    psi = inputs.gaussian_psi(shape, h, width=1.0, noise=1e-3, seed=seed)
    psi = psi + 1e-3j * inputs.random_psi(shape, seed=seed + 1).real
    return np.ascontiguousarray(psi)


SHAPES = [((8, 12, 16), 0.6), ((24, 18, 36), 0.35), ((32, 48, 24), 0.3)]


def test_boundary_roundtrip_keeps_48_bits():
    shape, h = (16, 12, 10), 0.5
    psi = state(shape, h)
    gpu = abi.Condensate(shape, h, 0.01, mode=abi.DGPE_REAL_TIME, precision=abi.DGPE_DF64)
    gpu.set_psi(psi)
    got = gpu.get_psi()
    assert got.dtype == np.complex128
    err = np.max(np.abs(got - psi) / np.maximum(np.abs(psi), 1e-300))
    assert err < 2.0 ** -47, err
    gpu.close()


@pytest.mark.parametrize("shape,h", SHAPES)
@pytest.mark.parametrize("mode", [abi.DGPE_REAL_TIME, abi.DGPE_IMAG_TIME])
def test_substeps_match_oracle(orc, shape, h, mode):
    psi = state(shape, h)
    gpu, p = make(orc, shape, h, 0.01, mode)
    for which, axis in [(abi.DGPE_SUB_CN_X, 0), (abi.DGPE_SUB_CN_Y, 1), (abi.DGPE_SUB_CN_Z, 2)]:
        gpu.set_psi(psi)
        gpu.substep(which)
        assert rel(gpu.get_psi(), orc.cn_sweep(p, psi, axis)) < DF_SUB_TOL, which
    gpu.set_psi(psi)
    gpu.substep(abi.DGPE_SUB_POTENTIAL)
    assert rel(gpu.get_psi(), orc.potential_step(p, psi)) < DF_SUB_TOL
    gpu.set_psi(psi)
    assert rel(gpu.phi(), orc.dipolar_phi(p, np.abs(psi) ** 2)) < DF_SUB_TOL
    gpu.close()


@pytest.mark.parametrize("shape,h", SHAPES + [((40, 28, 30), 0.3)])
@pytest.mark.parametrize("mode", [abi.DGPE_REAL_TIME, abi.DGPE_IMAG_TIME])
def test_full_steps_match_oracle(orc, shape, h, mode):
    psi = state(shape, h)
    gpu, p = make(orc, shape, h, 0.005, mode)
    gpu.set_psi(psi)
    gpu.step(12)
    assert rel(gpu.get_psi(), orc.step(p, psi, 12)) < DF_STEP_TOL
    gpu.close()


@pytest.mark.parametrize("shape", [(512, 6, 8), (6, 512, 8), (8, 6, 512)])
def test_longest_lines(orc, shape):
    """Lines of 512 points: the x and y sweeps fall back to the FP64 tile shape (the wide
    one does not fit in shared memory)."""
    psi = state(shape, 0.05)
    gpu, p = make(orc, shape, 0.05, 0.001, abi.DGPE_REAL_TIME)
    gpu.set_psi(psi)
    gpu.step(2)
    assert rel(gpu.get_psi(), orc.step(p, psi, 2)) < DF_STEP_TOL
    gpu.close()


@pytest.mark.parametrize("shape,h", SHAPES)
def test_observables_match_oracle(orc, shape, h):
    psi = state(shape, h)
    gpu, p = make(orc, shape, h, 0.01, abi.DGPE_IMAG_TIME)
    gpu.set_psi(psi)
    got, want = gpu.observables(), orc.observables(p, psi)
    for k in ("norm", "mu", "energy", "e_kin", "e_trap", "e_contact", "e_dipolar"):
        assert got[k] == pytest.approx(want[k], rel=1e-11, abs=1e-13), k
    gpu.close()


@pytest.mark.parametrize("dt", [3.0, -3.0, 0.37])
def test_large_phase_angles(orc, dt):
    """theta over many multiples of pi/2: the double-float argument reduction."""
    shape, h = (16, 12, 18), 0.6
    psi = state(shape, h)
    gpu, p = make(orc, shape, h, dt, abi.DGPE_REAL_TIME, nu=(2.0, 1.5, 2.5), g=40.0, gdd=30.0)
    gpu.set_psi(psi)
    gpu.substep(abi.DGPE_SUB_POTENTIAL)
    # theta up to ~500 carries 500 x 2^-48 of absolute error in a pair
    assert rel(gpu.get_psi(), orc.potential_step(p, psi)) < 1e-11
    gpu.close()


def test_imaginary_time_64cubed_200_steps(orc):
    shape, h = (64, 64, 64), 0.2
    psi0 = inputs.gaussian_psi(shape, h, noise=1e-3, seed=1)
    gpu, p = make(orc, shape, h, 0.004, abi.DGPE_IMAG_TIME, nu=(1, 1, 1), g=20, gdd=10)
    gpu.set_psi(psi0)
    gpu.step(200)
    want = orc.step(p, psi0, 200)
    assert rel(gpu.get_psi(), want) < DF_STEP_TOL
    og, ow = gpu.observables(), orc.observables(p, want)
    for k in ("norm", "mu", "energy"):
        assert og[k] == pytest.approx(ow[k], rel=1e-11)
    gpu.close()


def test_options_cutoff_simpson_radix5(orc):
    shape, h = (20, 28, 30), 0.35
    psi = state(shape, h)
    gpu, p = make(orc, shape, h, 0.005, abi.DGPE_IMAG_TIME, cutoff=3.1, integration=1, kinetic=1)
    gpu.set_psi(psi)
    gpu.step(6)
    want = orc.step(p, psi, 6)
    assert rel(gpu.get_psi(), want) < DF_STEP_TOL
    og, ow = gpu.observables(), orc.observables(p, want)
    for k in ("mu", "energy"):
        assert og[k] == pytest.approx(ow[k], rel=1e-10)
    gpu.close()


def test_matches_fp64_path_at_full_size():
    """256^3 real time, 20 steps from the same state: double-float against the FP64 path
    (both on the GPU)."""
    import torch
    shape, h = (256, 256, 256), 0.1
    psi = torch.from_numpy(inputs.gaussian_psi(shape, h, noise=1e-3, seed=1)).cuda()
    out = {}
    for prec in (abi.DGPE_FP64, abi.DGPE_DF64):
        gpu = abi.Condensate(shape, h, 5e-4, mode=abi.DGPE_REAL_TIME, precision=prec, nu=(0.5, 1.0, 1.5),
                             g=40.0, gdd=25.0)
        gpu.set_psi(psi)
        gpu.step(20)
        out[prec] = gpu.get_psi(host=False)
        gpu.close()
    a, b = out[abi.DGPE_DF64], out[abi.DGPE_FP64]
    assert float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) < 1e-11


def test_differentiation_is_unsupported():
    import torch
    shape, h = (16, 16, 16), 0.4
    gpu = abi.Condensate(shape, h, 0.01, mode=abi.DGPE_REAL_TIME, precision=abi.DGPE_DF64)
    z = torch.zeros(shape, dtype=torch.complex128, device="cuda")
    with pytest.raises(abi.DgpeError) as e:
        gpu.adjoint_step(z, z.clone())
    assert e.value.code == abi.DGPE_EUNSUPPORTED
    gpu.close()
