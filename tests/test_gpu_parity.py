"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the same
seeded inputs.  FP64 bar: relative L2 error of psi <= 1e-10 (the stated tolerance of the
FP64 path); sub-steps are held to 1e-12.  Shapes cover several tiles, ragged tails
(sizes that are not multiples of the 8/16-wide tiles), the smallest size 4 and the largest
line length 512 along each axis."""
import numpy as np
import pytest

from paper_1610_05329_gb300 import abi, inputs

pytestmark = pytest.mark.gpu

FP64_STEP_TOL = 1e-10
FP64_SUB_TOL = 1e-12


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1610_05329_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    abi.load()


def make(orc, shape, h, dt, mode, nu=(1.0, 1.1, 0.9), g=25.0, gdd=15.0, precision=abi.DGPE_FP64):
    gpu = abi.Condensate(shape, h, dt, mode=mode, precision=precision, nu=nu, g=g, gdd=gdd)
    p = orc.make_params(shape, h, dt, orc.IMAG_TIME if mode == abi.DGPE_IMAG_TIME else orc.REAL_TIME, nu, g, gdd)
    return gpu, p


def state(shape, h, seed=3):
    # a trapped-cloud shape plus seeded noise on both parts (every sub-step sees a complex field)
    psi = inputs.gaussian_psi(shape, h, width=1.0, noise=1e-3, seed=seed)
    psi = psi + 1e-3j * inputs.random_psi(shape, seed=seed + 1).real
    return np.ascontiguousarray(psi)


SHAPES = [((4, 6, 8), 0.9), ((8, 12, 16), 0.6), ((16, 16, 16), 0.5), ((24, 18, 36), 0.35),
          ((32, 48, 24), 0.3)]


@pytest.mark.parametrize("shape,h", SHAPES)
@pytest.mark.parametrize("mode", [abi.DGPE_REAL_TIME, abi.DGPE_IMAG_TIME])
def test_cn_sweeps_match_oracle(orc, shape, h, mode):
    psi = state(shape, h)
    gpu, p = make(orc, shape, h, 0.01, mode)
    for which, axis in [(abi.DGPE_SUB_CN_X, 0), (abi.DGPE_SUB_CN_Y, 1), (abi.DGPE_SUB_CN_Z, 2)]:
        gpu.set_psi(psi)
        gpu.substep(which)
        got = gpu.get_psi()
        want = orc.cn_sweep(p, psi, axis)
        assert rel(got, want) < FP64_SUB_TOL, (which, rel(got, want))
    gpu.close()


@pytest.mark.parametrize("shape,h", SHAPES)
def test_dipolar_potential_matches_oracle(orc, shape, h):
    psi = state(shape, h)
    gpu, p = make(orc, shape, h, 0.01, abi.DGPE_REAL_TIME)
    gpu.set_psi(psi)
    got = gpu.phi()
    want = orc.dipolar_phi(p, np.abs(psi) ** 2)
    assert rel(got, want) < FP64_SUB_TOL
    gpu.close()


@pytest.mark.parametrize("shape,h", SHAPES)
@pytest.mark.parametrize("mode", [abi.DGPE_REAL_TIME, abi.DGPE_IMAG_TIME])
def test_potential_step_matches_oracle(orc, shape, h, mode):
    psi = state(shape, h)
    gpu, p = make(orc, shape, h, 0.02, mode)
    gpu.set_psi(psi)
    gpu.substep(abi.DGPE_SUB_POTENTIAL)
    assert rel(gpu.get_psi(), orc.potential_step(p, psi)) < FP64_SUB_TOL
    gpu.close()


@pytest.mark.parametrize("shape,h", SHAPES)
def test_observables_match_oracle(orc, shape, h):
    psi = state(shape, h)
    gpu, p = make(orc, shape, h, 0.01, abi.DGPE_IMAG_TIME)
    gpu.set_psi(psi)
    got, want = gpu.observables(), orc.observables(p, psi)
    for k in ("norm", "mu", "energy", "e_kin", "e_trap", "e_contact", "e_dipolar"):
        assert got[k] == pytest.approx(want[k], rel=1e-11, abs=1e-13), k
    for d in range(3):
        assert got["rms"][d] == pytest.approx(want["rms"][d], rel=1e-11)
    gpu.close()


@pytest.mark.parametrize("shape,h", SHAPES)
@pytest.mark.parametrize("mode", [abi.DGPE_REAL_TIME, abi.DGPE_IMAG_TIME])
def test_full_steps_match_oracle(orc, shape, h, mode):
    psi = state(shape, h)
    gpu, p = make(orc, shape, h, 0.005, mode)
    gpu.set_psi(psi)
    gpu.step(12)
    got = gpu.get_psi()
    want = orc.step(p, psi, 12)
    assert rel(got, want) < FP64_STEP_TOL
    gpu.close()


@pytest.mark.parametrize("shape", [(512, 6, 8), (6, 512, 8), (8, 6, 512)])
def test_longest_lines(orc, shape):
    psi = state(shape, 0.05)
    gpu, p = make(orc, shape, 0.05, 0.001, abi.DGPE_REAL_TIME)
    gpu.set_psi(psi)
    gpu.step(2)
    assert rel(gpu.get_psi(), orc.step(p, psi, 2)) < FP64_STEP_TOL
    gpu.close()


@pytest.mark.parametrize("shape", [(150, 6, 8), (6, 300, 8), (8, 6, 384), (300, 10, 6)])
@pytest.mark.parametrize("precision,tol", [(abi.DGPE_FP64, FP64_STEP_TOL), (abi.DGPE_MIXED, 2e-5)])
def test_sweeps_on_lines_of_150_to_384(orc, shape, precision, tol):
    """Lines of 150, 300 and 384 points (partly filled lanes: 8 and 16 unknowns per lane,
    the last lanes idle)."""
    psi = state(shape, 0.05)
    cdt = np.complex128 if precision == abi.DGPE_FP64 else np.complex64
    gpu, p = make(orc, shape, 0.05, 0.001, abi.DGPE_REAL_TIME, precision=precision)
    gpu.set_psi(psi.astype(cdt))
    gpu.step(2)
    want = orc.step(p, psi.astype(cdt).astype(np.complex128), 2)
    assert rel(gpu.get_psi().astype(np.complex128), want) < tol
    gpu.close()


def test_imaginary_time_64cubed_200_steps(orc):
    """The 64^3 imaginary-time workload (h = 0.2, dt = 0.004, nu = 1, g = 20, gdd = 10,
    Gaussian + 1e-3 noise with seed 1, 200 steps) against the oracle: psi, mu, E, rms."""
    shape, h = (64, 64, 64), 0.2
    psi0 = inputs.gaussian_psi(shape, h, noise=1e-3, seed=1)
    gpu, p = make(orc, shape, h, 0.004, abi.DGPE_IMAG_TIME, nu=(1, 1, 1), g=20, gdd=10)
    gpu.set_psi(psi0)
    gpu.step(200)
    got = gpu.get_psi()
    want = orc.step(p, psi0, 200)
    assert rel(got, want) < FP64_STEP_TOL
    og, ow = gpu.observables(), orc.observables(p, want)
    for k in ("norm", "mu", "energy"):
        assert og[k] == pytest.approx(ow[k], rel=1e-11)
    gpu.close()


def test_set_params_quench_matches_oracle(orc):
    shape, h = (16, 24, 18), 0.45
    psi = state(shape, h)
    gpu, p_im = make(orc, shape, h, 0.01, abi.DGPE_IMAG_TIME)
    gpu.set_psi(psi)
    gpu.step(5)
    gpu.set_params(mode=abi.DGPE_REAL_TIME, dt=0.003, g=12.0)
    gpu.step(5)
    want = orc.step(p_im, psi, 5)
    p_re = orc.make_params(shape, h, 0.003, orc.REAL_TIME, (1.0, 1.1, 0.9), 12.0, 15.0)
    want = orc.step(p_re, want, 5)
    assert rel(gpu.get_psi(), want) < FP64_STEP_TOL
    gpu.close()


def test_device_psi_roundtrip_and_real_time_norm():
    import torch
    shape, h = (32, 32, 32), 0.3
    gpu = abi.Condensate(shape, h, 0.002, mode=abi.DGPE_REAL_TIME, nu=(1, 1, 1), g=30, gdd=10)
    psi = torch.from_numpy(inputs.gaussian_psi(shape, h, seed=5)).cuda()
    gpu.set_psi(psi)
    n0 = gpu.observables()["norm"]
    out = gpu.get_psi(host=False)
    # the first sweeps zero the walls; compare the norm after one step onwards
    gpu.step(1)
    n1 = gpu.observables()["norm"]
    gpu.step(100)
    n2 = gpu.observables()["norm"]
    assert abs(n2 - n1) < 1e-12 * n1
    assert torch.equal(out, psi)
    assert n0 > 0
    gpu.close()


def test_nonfinite_state_is_reported():
    shape, h = (16, 16, 16), 0.4
    gpu = abi.Condensate(shape, h, 0.01, mode=abi.DGPE_IMAG_TIME, g=10, gdd=5)
    psi = inputs.gaussian_psi(shape, h)
    psi[8, 8, 8] = np.nan
    gpu.set_psi(psi)
    gpu.step(1)
    with pytest.raises(abi.DgpeError) as e:
        gpu.sync()
    assert e.value.code == abi.DGPE_ENONFINITE
    # set_psi clears the latched error; the context stays usable
    gpu.set_psi(inputs.gaussian_psi(shape, h))
    gpu.step(1)
    gpu.sync()
    gpu.close()


@pytest.mark.parametrize("precision", [abi.DGPE_FP64, abi.DGPE_DF64, abi.DGPE_MIXED])
def test_zero_state(precision):
    """The degenerate state psi = 0: real time keeps it exactly zero with no error;
    imaginary time cannot renormalise it and reports DGPE_ENONFINITE, as do the observables
    (mu = E / norm is undefined)."""
    shape, h = (12, 10, 8), 0.5
    dtype = np.complex64 if precision == abi.DGPE_MIXED else np.complex128
    zero = np.zeros(shape, dtype)
    gpu = abi.Condensate(shape, h, 0.01, mode=abi.DGPE_REAL_TIME, precision=precision, g=10, gdd=5)
    gpu.set_psi(zero)
    gpu.step(3)
    gpu.sync()
    assert not np.any(gpu.get_psi())
    with pytest.raises(abi.DgpeError) as e:
        gpu.observables()
    assert e.value.code == abi.DGPE_ENONFINITE
    gpu.close()
    gpu = abi.Condensate(shape, h, 0.01, mode=abi.DGPE_IMAG_TIME, precision=precision, g=10, gdd=5)
    gpu.set_psi(zero)
    gpu.step(1)
    with pytest.raises(abi.DgpeError) as e:
        gpu.sync()
    assert e.value.code == abi.DGPE_ENONFINITE
    gpu.close()


@pytest.mark.parametrize("mode", [abi.DGPE_REAL_TIME, abi.DGPE_IMAG_TIME])
def test_mixed_precision_error_vs_oracle(orc, mode):
    """FP32 path (complex64 psi, FP32 FFT/phase/CN, FP64 reductions): errors against the
    FP64 oracle after 20 steps.  Bounds: FP32 round-off (6e-8) times the step count and
    the transform depth, with margin."""
    shape, h = (32, 24, 36), 0.3
    psi = state(shape, h)
    gpu, p = make(orc, shape, h, 0.005, mode, precision=abi.DGPE_MIXED)
    gpu.set_psi(psi.astype(np.complex64))
    gpu.step(20)
    got = gpu.get_psi().astype(np.complex128)
    want = orc.step(p, psi.astype(np.complex64).astype(np.complex128), 20)
    err = rel(got, want)
    assert err < 2e-5, err
    og, ow = gpu.observables(), orc.observables(p, want)
    assert og["mu"] == pytest.approx(ow["mu"], rel=2e-5)
    assert og["energy"] == pytest.approx(ow["energy"], rel=2e-5)
    gpu.close()


@pytest.mark.parametrize("mode", [abi.DGPE_IMAG_TIME, abi.DGPE_REAL_TIME])
@pytest.mark.parametrize("shape", [(48, 64, 20), (96, 128, 12), (128, 32, 36), (32, 48, 128), (20, 24, 96),
                                   (24, 20, 64)])
def test_mixed_short_line_sweeps_vs_oracle(orc, shape, mode):
    """x and y lines of 32, 48, 64, 96 and 128 points take the 8-lane sweeps (4, 6, 8, 12 and
    16 points per lane), with nz not a multiple of the 16-column tiles; z lines of 64, 96 and
    128 the 8-lane solve inside K5: FP32 errors against the FP64 oracle after 10 steps, at
    the FP32-mixed bar of the 20-step test."""
    h = 0.25
    psi = state(shape, h)
    gpu, p = make(orc, shape, h, 0.004, mode, precision=abi.DGPE_MIXED)
    gpu.set_psi(psi.astype(np.complex64))
    gpu.step(10)
    got = gpu.get_psi().astype(np.complex128)
    want = orc.step(p, psi.astype(np.complex64).astype(np.complex128), 10)
    assert rel(got, want) < 2e-5
    og, ow = gpu.observables(), orc.observables(p, want)
    assert og["mu"] == pytest.approx(ow["mu"], rel=2e-5)
    assert og["rms"][0] == pytest.approx(ow["rms"][0], rel=2e-5)
    gpu.close()


@pytest.mark.parametrize("dt", [3.0, -3.0, 0.37])
def test_potential_step_large_phase_angles(orc, dt):
    """theta = dt (V + g n + gdd Phi) spanning many multiples of pi/2 (both signs), which
    exercises the argument reduction of the FP64 sine/cosine."""
    shape, h = (16, 12, 18), 0.6
    psi = state(shape, h)
    gpu, p = make(orc, shape, h, dt, abi.DGPE_REAL_TIME, nu=(2.0, 1.5, 2.5), g=40.0, gdd=30.0)
    gpu.set_psi(psi)
    gpu.substep(abi.DGPE_SUB_POTENTIAL)
    assert rel(gpu.get_psi(), orc.potential_step(p, psi)) < FP64_SUB_TOL
    gpu.close()


@pytest.mark.parametrize("dt", [3.0, -3.0, 0.37, 0.004])
def test_potential_step_large_phase_angles_fp32(orc, dt):
    """The FP32 sine/cosine (three-float pi/2 reduction, Taylor series) over angles up to a
    few hundred radians of both signs.  Bound: theta is formed in FP32 from four rounded
    terms (a few ulp of |theta|max), then reduced and evaluated to ~1e-7."""
    shape, h, nu, g, gdd = (16, 12, 18), 0.6, (2.0, 1.5, 2.5), 40.0, 30.0
    psi = state(shape, h).astype(np.complex64).astype(np.complex128)
    gpu, p = make(orc, shape, h, dt, abi.DGPE_REAL_TIME, nu=nu, g=g, gdd=gdd, precision=abi.DGPE_MIXED)
    gpu.set_psi(psi.astype(np.complex64))
    gpu.substep(abi.DGPE_SUB_POTENTIAL)
    got = gpu.get_psi().astype(np.complex128)
    want = orc.potential_step(p, psi)
    x, y, z = inputs.grid_axes(shape, (h, h, h))
    vmax = 0.5 * (nu[0] ** 2 * np.max(x ** 2) + nu[1] ** 2 * np.max(y ** 2) + nu[2] ** 2 * np.max(z ** 2))
    n = np.abs(psi) ** 2
    theta_max = abs(dt) * (vmax + g * n.max() + gdd * np.abs(orc.dipolar_phi(p, n)).max())
    assert theta_max > 1.0 or dt == 0.004
    assert rel(got, want) < 5e-7 * theta_max + 1e-6, (rel(got, want), theta_max)
    gpu.close()


@pytest.mark.parametrize("shape,h", [((10, 20, 14), 0.5), ((40, 28, 30), 0.3), ((70, 10, 50), 0.25)])
@pytest.mark.parametrize("mode", [abi.DGPE_REAL_TIME, abi.DGPE_IMAG_TIME])
def test_radix5_radix7_sizes(orc, shape, h, mode):
    """Grid sizes with factors 5 and 7 (the paper's FFT-friendly sizes 2^a 3^b 5^c 7^d)."""
    psi = state(shape, h)
    gpu, p = make(orc, shape, h, 0.005, mode)
    gpu.set_psi(psi)
    assert rel(gpu.phi(), orc.dipolar_phi(p, np.abs(psi) ** 2)) < FP64_SUB_TOL
    gpu.step(6)
    assert rel(gpu.get_psi(), orc.step(p, psi, 6)) < FP64_STEP_TOL
    gpu.close()


@pytest.mark.parametrize("precision,tol", [(abi.DGPE_FP64, FP64_STEP_TOL), (abi.DGPE_MIXED, 2e-5)])
def test_spherical_cutoff(orc, precision, tol):
    """Dipolar interaction restricted to r < R (R = 3.1, inside the box of 9.6)."""
    shape, h, R = (24, 32, 36), (0.4, 0.3, 0.27), 3.1
    psi = state(shape, h)
    gpu = abi.Condensate(shape, h, 0.005, mode=abi.DGPE_REAL_TIME, precision=precision, nu=(1.0, 1.1, 0.9),
                         g=25.0, gdd=15.0, cutoff=R)
    p = orc.make_params(shape, h, 0.005, orc.REAL_TIME, (1.0, 1.1, 0.9), 25.0, 15.0, cutoff=R)
    cdt = np.complex128 if precision == abi.DGPE_FP64 else np.complex64
    gpu.set_psi(psi.astype(cdt))
    want_phi = orc.dipolar_phi(p, np.abs(psi.astype(cdt).astype(np.complex128)) ** 2)
    assert rel(gpu.phi(), want_phi) < (FP64_SUB_TOL if precision == abi.DGPE_FP64 else 1e-5)
    gpu.step(8)
    want = orc.step(p, psi.astype(cdt).astype(np.complex128), 8)
    assert rel(gpu.get_psi().astype(np.complex128), want) < tol
    gpu.close()


@pytest.mark.parametrize("integration,kinetic", [(1, 0), (0, 1), (1, 1)])
def test_simpson_and_gradient_observables(orc, integration, kinetic):
    """The quadrature/derivative options: imaginary-time steps renormalised with Simpson
    weights, and the observables with Simpson weights and/or the 5-point gradient."""
    shape, h = (24, 18, 36), 0.35
    psi = state(shape, h)
    gpu = abi.Condensate(shape, h, 0.005, mode=abi.DGPE_IMAG_TIME, nu=(1.0, 1.1, 0.9), g=25.0, gdd=15.0,
                         integration=integration, kinetic=kinetic)
    p = orc.make_params(shape, h, 0.005, orc.IMAG_TIME, (1.0, 1.1, 0.9), 25.0, 15.0, integration=integration,
                        kinetic=kinetic)
    gpu.set_psi(psi)
    gpu.step(10)
    got, want = gpu.get_psi(), orc.step(p, psi, 10)
    assert rel(got, want) < FP64_STEP_TOL
    og, ow = gpu.observables(), orc.observables(p, want)
    for k in ("norm", "mu", "energy", "e_kin"):
        assert og[k] == pytest.approx(ow[k], rel=1e-11), k
    for d in range(3):
        assert og["rms"][d] == pytest.approx(ow["rms"][d], rel=1e-11)
    assert og["norm"] == pytest.approx(1.0, abs=1e-12)
    gpu.close()


@pytest.mark.parametrize("precision,tol", [(abi.DGPE_FP64, FP64_STEP_TOL), (abi.DGPE_MIXED, 2e-5)])
def test_compile_time_transforms_match_runtime_plans(orc, precision, tol):
    """Lengths 128 and 256 with the default radix order run the compile-time transforms (K1,
    K2, K3, K4 and K5's step); the radix-4-first and radix-3-first orders run the runtime
    plans.  Both agree with the oracle after three real-time steps."""
    shape, h, dt = (128, 128, 256), 0.12, 0.002
    cdt = np.complex128 if precision == abi.DGPE_FP64 else np.complex64
    psi = state(shape, h).astype(cdt)
    gpu, p = make(orc, shape, h, dt, abi.DGPE_REAL_TIME, precision=precision)
    want = orc.step(p, psi.astype(np.complex128), 3)
    default = gpu.tuning()
    assert default["plan_style"] == (0, 0, 0) and default["fft_threads"] == 256
    got = {}
    for style in (0, 1, 2):
        gpu.set_tuning(dict(default, plan_style=(style, style, style)))
        gpu.set_psi(psi)
        gpu.step(3)
        got[style] = gpu.get_psi().astype(np.complex128)
        assert rel(got[style], want) < tol, (style, rel(got[style], want))
    assert rel(got[0], got[1]) < tol and rel(got[0], got[2]) < tol
    gpu.close()


def test_step_launches():
    """Seven kernels per step, eight where the z sweep is a pass of its own (FP64)."""
    for prec, want in ((abi.DGPE_FP64, 8), (abi.DGPE_DF64, 8), (abi.DGPE_MIXED, 7)):
        gpu = abi.Condensate((16, 16, 16), 0.5, 0.01, mode=abi.DGPE_REAL_TIME, precision=prec)
        assert gpu.step_launches() == want
        gpu.close()
