"""The seeded generator shared by both sides: SplitMix64 against its published outputs."""
import numpy as np

from paper_1610_05329_gb300 import inputs


def test_splitmix64_reference_outputs():
    # First outputs of SplitMix64 with seed 0 (the reference C implementation's sequence).
    got = inputs.splitmix64(0, 3)
    assert [int(v) for v in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_range_and_determinism():
    a = inputs.uniform(1, 100000, -1e-3, 1e-3)
    assert a.min() >= -1e-3 and a.max() < 1e-3
    assert abs(a.mean()) < 1e-5
    assert np.array_equal(a, inputs.uniform(1, 100000, -1e-3, 1e-3))


def test_gaussian_psi_continuum_normalised():
    psi = inputs.gaussian_psi((64, 64, 64), 0.2, noise=0)
    assert abs(np.sum(np.abs(psi) ** 2) * 0.2 ** 3 - 1) < 1e-12
    assert psi.flags["C_CONTIGUOUS"] and psi.dtype == np.complex128
