"""dgpe_step_host: host-resident states through the solver with the copies of successive
calls overlapped with the steps.  Each call must give exactly what the synchronous
dgpe_set_psi / dgpe_step / dgpe_get_psi sequence gives (the same kernels on the same data),
and the FP64 result matches the oracle."""
import numpy as np
import pytest

from paper_1610_05329_gb300 import abi, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1610_05329_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    abi.load()


def states(shape, h, dtype, k):
    out = []
    for q in range(k):
        psi = inputs.gaussian_psi(shape, h, width=1.0 + 0.1 * q, noise=1e-3, seed=10 + q)
        out.append(np.ascontiguousarray(psi.astype(dtype)))
    return out


@pytest.mark.parametrize("precision", [abi.DGPE_FP64, abi.DGPE_DF64, abi.DGPE_MIXED])
@pytest.mark.parametrize("mode", [abi.DGPE_REAL_TIME, abi.DGPE_IMAG_TIME])
def test_pipelined_calls_match_synchronous_calls(precision, mode):
    import torch
    shape, h = (24, 20, 30), 0.4
    kw = dict(mode=mode, precision=precision, nu=(1.0, 1.2, 0.8), g=30.0, gdd=12.0)
    ref = abi.Condensate(shape, h, 0.005, **kw)
    io = abi.Condensate(shape, h, 0.005, **kw)
    dtype = np.complex64 if precision == abi.DGPE_MIXED else np.complex128
    tdtype = torch.complex64 if precision == abi.DGPE_MIXED else torch.complex128
    tol = 1e-5 if precision == abi.DGPE_MIXED else 1e-12
    ins = states(shape, h, dtype, 4)
    want = []
    for a in ins:
        ref.set_psi(a)
        ref.step(3)
        want.append(ref.get_psi())
    pin_in = [torch.from_numpy(a).pin_memory() for a in ins]
    pin_out = [torch.empty(shape, dtype=tdtype).pin_memory() for _ in ins]
    for a, b in zip(pin_in, pin_out):   # four calls in flight before the one sync
        io.step_host(a, b, 3)
    io.sync()
    for q in range(len(ins)):
        assert np.array_equal(pin_out[q].numpy(), want[q]), q
    # the same output buffer reused by consecutive calls holds the last result
    same = torch.empty(shape, dtype=tdtype).pin_memory()
    for a in pin_in:
        io.step_host(a, same, 3)
    io.sync()
    assert np.array_equal(same.numpy(), want[-1])
    # the state stays on the context: plain steps continue from it (whichever of the two
    # buffers holds it), and a parameter change rebuilds the captured step of both buffers
    for extra in range(2):
        io.step_host(pin_in[extra], pin_out[extra], 3)
        io.step(2)            # waits for the output copy, which reads the state buffer
        ref.set_psi(ins[extra])
        ref.step(5)
        # imaginary time: the output applies the pending renormalisation to the state after
        # 3 steps, which rounds differently from applying it after 5
        got, exp = io.get_psi(), ref.get_psi()
        assert np.linalg.norm(got - exp) <= tol * np.linalg.norm(exp), extra
        io.sync()
        assert np.array_equal(pin_out[extra].numpy(), want[extra]), extra
    for c in (io, ref):
        c.set_params(g=20.0)
    io.step_host(pin_in[0], pin_out[0], 3)
    io.sync()
    ref.set_psi(ins[0])
    ref.step(3)
    assert np.array_equal(pin_out[0].numpy(), ref.get_psi())
    ref.close()
    io.close()


def test_fp64_matches_oracle(orc):
    import torch
    shape, h = (32, 24, 28), 0.35
    psi = states(shape, h, np.complex128, 1)[0]
    gpu = abi.Condensate(shape, h, 0.004, mode=abi.DGPE_REAL_TIME, precision=abi.DGPE_FP64, nu=(1, 1, 1),
                         g=20.0, gdd=10.0)
    p = orc.make_params(shape, h, 0.004, orc.REAL_TIME, (1, 1, 1), 20.0, 10.0)
    src = torch.from_numpy(psi).pin_memory()
    dst = torch.empty(shape, dtype=torch.complex128).pin_memory()
    gpu.step_host(src, dst, 5)
    gpu.sync()
    want = orc.step(p, psi, 5)
    assert np.linalg.norm(dst.numpy() - want) / np.linalg.norm(want) < 1e-10
    gpu.close()


def test_invalid_arguments():
    shape = (8, 8, 8)
    gpu = abi.Condensate(shape, 0.5, 0.01, mode=abi.DGPE_REAL_TIME, precision=abi.DGPE_FP64)
    with pytest.raises(abi.DgpeError) as e:
        abi.dgpe_step_host(gpu.ctx, 0, 0, 1)
    assert e.value.code == abi.DGPE_EINVAL
    buf = np.zeros(shape, np.complex128)
    with pytest.raises(abi.DgpeError) as e:
        abi.dgpe_step_host(gpu.ctx, buf.ctypes.data, buf.ctypes.data, -1)
    assert e.value.code == abi.DGPE_EINVAL
    gpu.close()
