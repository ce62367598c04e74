"""Pins of the oracle's transforms (recursive Cooley-Tukey, naive DFT, 3D row-column).

The dipolar term is evaluated "by a Fourier transformation to momentum space" (paper,
Solution method); the oracle's own FFT is pinned here against closed forms of the DFT,
the naive O(n^2) sum, an independent library FFT (numpy.fft), Parseval and inversion.
"""
import numpy as np
import pytest

from paper_1610_05329_gb300 import inputs

SIZES = [1, 2, 3, 4, 6, 8, 9, 12, 16, 18, 24, 27, 32, 48, 64, 96, 128, 384]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_dft_closed_forms(orc):
    # DFT of a unit impulse at j0 is exp(-2 pi i k j0 / n); of exp(+2 pi i m j / n) it is n delta_km.
    for n in (5, 6, 8, 12):
        j = np.arange(n)
        for j0 in range(n):
            x = np.zeros(n, complex)
            x[j0] = 1
            assert np.allclose(orc.dft(x), np.exp(-2j * np.pi * j * j0 / n), atol=1e-14)
        for m in range(n):
            x = np.exp(2j * np.pi * m * j / n)
            want = np.zeros(n, complex)
            want[m] = n
            assert np.allclose(orc.dft(x), want, atol=1e-12)
            assert np.allclose(orc.dft(np.conj(x), +1), np.conj(want), atol=1e-12)


@pytest.mark.parametrize("n", SIZES)
def test_fft_equals_naive_dft(orc, n):
    x = inputs.random_psi((n,), seed=n)
    for sign in (-1, 1):
        assert rel(orc.fft(x, sign), orc.dft(x, sign)) < 1e-13


@pytest.mark.parametrize("n", SIZES)
def test_fft_matches_numpy(orc, n):
    x = inputs.random_psi((n,), seed=100 + n)
    assert rel(orc.fft(x, -1), np.fft.fft(x)) < 1e-13
    assert rel(orc.fft(x, +1), n * np.fft.ifft(x)) < 1e-13


@pytest.mark.parametrize("n", [6, 16, 48, 384])
def test_parseval_and_inverse(orc, n):
    x = inputs.random_psi((n,), seed=3 * n)
    X = orc.fft(x, -1)
    assert abs(np.vdot(X, X).real - n * np.vdot(x, x).real) < 1e-12 * n * np.vdot(x, x).real
    assert rel(orc.fft(X, +1) / n, x) < 1e-14


def test_real_input_hermitian(orc):
    # Real input => X[n-k] = conj(X[k]); the R2C half spectrum is the first n/2+1 bins.
    for n in (8, 12, 48):
        x = inputs.uniform(n, n, -1, 1).astype(complex)
        X = orc.fft(x, -1)
        k = np.arange(1, n)
        assert np.allclose(X[n - k], np.conj(X[k]), atol=1e-13)
        assert abs(X[0].imag) < 1e-13 and abs(X[n // 2].imag) < 1e-13


@pytest.mark.parametrize("shape", [(4, 6, 8), (6, 6, 6), (8, 12, 16), (16, 24, 32)])
def test_fft3_matches_numpy(orc, shape):
    x = inputs.random_psi(shape, seed=11)
    assert rel(orc.fft3(x, -1), np.fft.fftn(x)) < 1e-13
    assert rel(orc.fft3(orc.fft3(x, -1), +1) / x.size, x) < 1e-14
