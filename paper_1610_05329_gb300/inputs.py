"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the CPU oracle.

This module holds no arithmetic of the SSCN method: it only draws initial wave functions.
Both sides receive the same arrays, so neither side's inputs come from the other.

Noise generator: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), state_i = seed + (i + 1) * 0x9E3779B97F4A7C15, then the
published three-stage mix; doubles take the top 53 bits: u = (z >> 11) * 2^-53 in [0, 1).
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, count):
    """The first `count` outputs of SplitMix64 seeded with `seed` (uint64 array)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, count, lo=0.0, hi=1.0):
    """`count` doubles uniform in [lo, hi) from SplitMix64(seed), 53-bit mantissa."""
    u = (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def grid_axes(shape, h):
    """Coordinates x_i = (i - N/2) h of each axis (the grid convention of the solver)."""
    hs = (h, h, h) if np.isscalar(h) else tuple(h)
    return [(np.arange(n, dtype=np.float64) - n // 2) * hh for n, hh in zip(shape, hs)]


def gaussian_psi(shape, h, width=1.0, noise=1e-3, seed=1, center=(0.0, 0.0, 0.0)):
    """pi^{-3/4} w^{-3/2} exp(-|r - c|^2 / (2 w^2)) + U[-noise, noise) added to Re psi.

    The Gaussian is normalised in the continuum (width w = 1 gives pi^{-3/4} e^{-r^2/2});
    the noise is drawn in row-major [nx][ny][nz] order from SplitMix64(seed).
    Returns a C-contiguous complex128 array of the given shape.
    """
    x, y, z = grid_axes(shape, h)
    r2 = ((x[:, None, None] - center[0]) ** 2 + (y[None, :, None] - center[1]) ** 2
          + (z[None, None, :] - center[2]) ** 2)
    psi = (np.pi ** -0.75) * width ** -1.5 * np.exp(-r2 / (2.0 * width * width))
    psi = psi.astype(np.complex128)
    if noise:
        n = int(np.prod(shape))
        psi.real += uniform(seed, n, -noise, noise).reshape(shape)
    return np.ascontiguousarray(psi)


def random_psi(shape, seed=7, scale=1.0):
    """Complex field with independent U[-scale, scale) real and imaginary parts (tests of
    linear sub-steps, where no physical shape is needed)."""
    n = int(np.prod(shape))
    re = uniform(seed, n, -scale, scale)
    im = uniform(seed + 0x5bd1e995, n, -scale, scale)
    return np.ascontiguousarray((re + 1j * im).reshape(shape))
