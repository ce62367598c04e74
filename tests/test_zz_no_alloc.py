"""dgpe_moments_noalloc: the allocation-free norm/rms call against dgpe_observables.

Some callers cannot allocate device memory while they run (their framework owns every
byte through its own pool, or a cudaMalloc inside a time-critical loop would synchronise
the device); this call serves them with a fixed scratch array inside the library.  It must
give the same norm and rms sizes as the context-based observables call, on two calls in a
row (the second finds the scratch left over by the first).  This file is collected last so
that a run stopping at its first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1610_05329_gb300 import abi, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("integration", [abi.DGPE_RECTANGLE, abi.DGPE_SIMPSON])
@pytest.mark.parametrize("precision", [abi.DGPE_FP64, abi.DGPE_MIXED, abi.DGPE_DF64])
def test_moments_noalloc_matches_observables(precision, integration):
    """Same norm and rms sizes as dgpe_observables of a context in the same precision and
    quadrature (the double-float mode hands complex128 states to its callers)."""
    import torch
    from paper_1610_05329_gb300 import build
    build.build()
    shape, h = (24, 36, 48), (0.3, 0.25, 0.2)
    gpu = abi.Condensate(shape, h, 0.01, mode=abi.DGPE_IMAG_TIME, precision=precision, nu=(1.0, 1.3, 0.8),
                         g=20.0, gdd=10.0, integration=integration)
    psi = inputs.gaussian_psi(shape, h, width=1.1, noise=1e-3, seed=17, center=(0.3, -0.2, 0.1))
    gpu.set_psi(psi)
    gpu.step(3)                       # a state with a pending renormalisation
    want = gpu.observables()
    dev_psi = gpu.get_psi(host=False)  # the normalised state, in device memory
    out = torch.zeros(4, dtype=torch.float64, device=dev_psi.device)
    params = abi.make_params(shape, h, 0.01, precision=precision, integration=integration)
    tol = 1e-6 if precision == abi.DGPE_MIXED else 1e-11
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out.zero_()
        abi.dgpe_moments_noalloc(dev_psi.data_ptr(), params, out.data_ptr(), stream)
        got = out.cpu().numpy()
        assert got[0] == pytest.approx(want["norm"], rel=tol)
        for d in range(3):
            assert got[1 + d] == pytest.approx(want["rms"][d], rel=tol)
    gpu.close()


def test_moments_noalloc_rejects_bad_sizes():
    import torch
    from paper_1610_05329_gb300 import build
    build.build()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    psi = torch.zeros(8, dtype=torch.complex128, device="cuda")
    too_big = abi.make_params((1024, 512, 512), 0.1, 0.01)
    with pytest.raises(abi.DgpeError) as e:
        abi.dgpe_moments_noalloc(psi.data_ptr(), too_big, out.data_ptr())
    assert e.value.code == abi.DGPE_EUNSUPPORTED
    with pytest.raises(abi.DgpeError) as e:
        abi.dgpe_moments_noalloc(psi.data_ptr(), abi.make_params((2, 2, 2), 0.0, 0.01), out.data_ptr())
    assert e.value.code == abi.DGPE_EINVAL
