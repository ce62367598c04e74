"""Pins of the oracle's dipolar mean field Phi = IDFT[Ut(k) DFT(n)], Ut = 3 kz^2/k^2 - 1.

The paper evaluates the dipolar term in momentum space, where the convolution with the
dipolar interaction becomes a product (Solution method).  Pins:
  * brute force: the FFT path equals the direct circular convolution with the real-space
    kernel K = naive IDFT(Ut) on tiny grids;
  * closed form: for a cylindrical Gaussian density the dipolar energy 1/2 int Phi n equals
    -f(kappa) / (2 (2 pi)^{3/2} s_rho^2 s_z) (Lahaye et al., Rep. Prog. Phys. 72, 126401
    (2009)), f the anisotropy function, for both kappa < 1 and kappa > 1; the closed form is
    itself checked against an independent 1D quadrature of the k-space integral;
  * symmetry: an isotropic density has zero dipolar energy on a cubic grid;
  * anisotropic grids: the kernel's values at hand-derived wavenumbers on a grid whose three
    axes differ in both N and h (box lengths 4, 6 and 3, so no two axes share a wavenumber
    spacing), and the closed-form energy on a grid with unequal N and h per axis.
"""
import numpy as np
import pytest
from scipy import integrate


def f_kappa(k):
    """Anisotropy function of the dipolar energy of a Gaussian (kappa = s_rho / s_z)."""
    if k < 1:
        s = np.sqrt(1 - k * k)
        return (1 + 2 * k * k) / (1 - k * k) - 3 * k * k * np.arctanh(s) / (1 - k * k) ** 1.5
    s = np.sqrt(k * k - 1)
    return (1 + 2 * k * k) / (1 - k * k) + 3 * k * k * np.arctan(s) / (k * k - 1) ** 1.5


def e_dd_closed(sr, sz):
    return -f_kappa(sr / sz) / (2 * (2 * np.pi) ** 1.5 * sr * sr * sz)


def e_dd_quadrature(sr, sz):
    # 1/2 int d^3k/(2 pi)^3 (3 cos^2 a - 1) exp(-(k_rho^2 sr^2 + k_z^2 sz^2)/2); the radial
    # integral int k^2 exp(-k^2 A/2) dk = sqrt(pi/2) A^{-3/2} is done analytically.
    def integrand(u):
        a = (1 - u * u) * sr * sr + u * u * sz * sz
        return (3 * u * u - 1) * np.sqrt(np.pi / 2) * a ** -1.5
    val, _ = integrate.quad(integrand, -1, 1, epsabs=1e-15, epsrel=1e-13, limit=200)
    return 0.5 * 2 * np.pi * val / (2 * np.pi) ** 3


def gaussian_density(shape, h, sr, sz):
    axes = [(np.arange(n) - n // 2) * hd for n, hd in zip(shape, h)]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    return np.exp(-(X ** 2 + Y ** 2) / sr ** 2 - Z ** 2 / sz ** 2) / (np.pi ** 1.5 * sr * sr * sz)


def grid_e_dd(orc, n, h, sr, sz):
    """1/2 h^3 sum Phi n of the cylindrical Gaussian; n and h per axis (or one for all)."""
    shape = (n, n, n) if np.isscalar(n) else tuple(n)
    hs = (h, h, h) if np.isscalar(h) else tuple(h)
    p = orc.make_params(shape, hs, 1e-3, orc.REAL_TIME, (1, 1, 1), 0.0, 1.0)
    dens = gaussian_density(shape, hs, sr, sz)
    return 0.5 * np.sum(orc.dipolar_phi(p, dens) * dens) * np.prod(hs)


def test_kernel_geometry(orc):
    # Ut = 3 cos^2(angle to z) - 1: +2 along the dipole axis, -1 perpendicular, 0 at k = 0.
    p = orc.make_params((8, 8, 8), 0.5, 1e-3, orc.REAL_TIME, (1, 1, 1), 0, 1)
    ut = orc.dipolar_kernel(p)
    assert ut[0, 0, 0] == 0.0
    assert ut[0, 0, 1] == pytest.approx(2.0) and ut[0, 0, 7] == pytest.approx(2.0)
    assert ut[1, 0, 0] == pytest.approx(-1.0) and ut[0, 3, 0] == pytest.approx(-1.0)
    assert ut[1, 0, 1] == pytest.approx(0.5)          # 45 degrees: 3/2 - 1
    assert np.array_equal(ut, ut[::-1, ::-1, ::-1][np.ix_(*[np.roll(np.arange(8), 1)] * 3)])  # even


# Anisotropic grid: nx = 8, hx = 0.5 (box 4), ny = 12, hy = 0.5 (box 6), nz = 12, hz = 0.25
# (box 3), so k_x = pi m/2, k_y = pi m/3, k_z = 2 pi m/3 for the signed index m.  Values of
# Ut = 3 kz^2/|k|^2 - 1 worked out by hand at these indices:
#   (4, 0, 3): kx = 2 pi (the Nyquist index, m = +4), kz = 2 pi       -> 45 degrees: 1/2
#   (0, 2, 1): ky = 2 pi/3, kz = 2 pi/3                               -> 1/2
#   (0, 0, 5): along z                                                -> 2
#   (3, 0, 0), (0, 5, 0): in the xy plane                             -> -1
#   (1, 1, 1): |k|^2 = pi^2 (1/4 + 1/9 + 4/9) = 29 pi^2/36, kz^2 = 16 pi^2/36 -> 48/29 - 1 = 19/29
#   (7, 11, 11): the signed indices (-1, -1, -1)                      -> 19/29
#   (2, 3, 1): |k|^2 = pi^2 (1 + 1 + 4/9) = 22 pi^2/9, kz^2 = 4 pi^2/9  -> 12/22 - 1 = -5/11
ANISO_GRID = ((8, 12, 12), (0.5, 0.5, 0.25))
ANISO_PINS = {(4, 0, 3): 0.5, (0, 2, 1): 0.5, (0, 0, 5): 2.0, (3, 0, 0): -1.0, (0, 5, 0): -1.0,
              (1, 1, 1): 19 / 29, (7, 11, 11): 19 / 29, (2, 3, 1): -5 / 11}


def test_kernel_geometry_anisotropic(orc):
    shape, h = ANISO_GRID
    ut = orc.dipolar_kernel(orc.make_params(shape, h, 1e-3, orc.REAL_TIME, (1, 1, 1), 0, 1))
    assert ut.shape == shape
    assert ut[0, 0, 0] == 0.0
    for idx, want in ANISO_PINS.items():
        assert ut[idx] == pytest.approx(want, rel=1e-14, abs=1e-15), idx


def test_anisotropic_pins_detect_axis_mixups():
    """The pins above fail if any axis's N or h is taken from another axis: every other
    assignment of the (N, h) pairs to the axes, and every swap of one axis's h with another
    axis's, changes at least one pinned value (the values evaluated here by hand formula,
    not by the oracle; this shows the pins discriminate, it pins nothing itself)."""
    import itertools
    shape, h = ANISO_GRID

    def ut_at(idx, ns, hs):
        k = []
        for m, n, hd in zip(idx, ns, hs):
            ms = m if m <= n // 2 else m - n
            k.append(2 * np.pi * ms / (n * hd))
        k2 = sum(v * v for v in k)
        return 3 * k[2] ** 2 / k2 - 1 if k2 > 0 else 0.0

    def pins_hold(ns, hs):
        return all(abs(ut_at(idx, ns, hs) - want) < 1e-9 for idx, want in ANISO_PINS.items())

    assert pins_hold(shape, h)
    for perm in itertools.permutations(range(3)):
        if perm != (0, 1, 2):
            assert not pins_hold([shape[a] for a in perm], [h[a] for a in perm]), perm
    for a, b in itertools.combinations(range(3), 2):
        hs = list(h)
        hs[a], hs[b] = hs[b], hs[a]
        ns = list(shape)
        ns[a], ns[b] = ns[b], ns[a]
        if hs != list(h):
            assert not pins_hold(shape, hs), ("h", a, b)
        if ns != list(shape):
            assert not pins_hold(ns, h), ("n", a, b)


@pytest.mark.parametrize("shape,h", [((4, 6, 8), (0.5, 0.4, 0.3)), ((6, 6, 6), 0.7), ((8, 4, 6), (0.3, 0.9, 0.5))])
def test_fft_convolution_equals_direct(orc, shape, h):
    from paper_1610_05329_gb300 import inputs
    p = orc.make_params(shape, h, 1e-3, orc.REAL_TIME, (1, 1, 1), 0, 1)
    n = inputs.uniform(5, int(np.prod(shape)), 0, 1).reshape(shape)
    phi_fft = orc.dipolar_phi(p, n)
    phi_dir = orc.dipolar_phi_direct(p, n)
    assert np.max(np.abs(phi_fft - phi_dir)) < 1e-13 * np.max(np.abs(phi_dir))


@pytest.mark.parametrize("sr,sz", [(1.0, 0.6), (0.6, 1.0)])
def test_closed_form_is_the_integral(sr, sz):
    assert e_dd_closed(sr, sz) == pytest.approx(e_dd_quadrature(sr, sz), rel=1e-12)


@pytest.mark.parametrize("sr,sz", [(1.0, 0.6), (0.6, 1.0)])
def test_gaussian_dipolar_energy(orc, sr, sz):
    exact = e_dd_closed(sr, sz)
    small = grid_e_dd(orc, 32, 0.3, sr, sz)   # box 9.6
    large = grid_e_dd(orc, 64, 0.3, sr, sz)   # box 19.2
    assert np.sign(large) == np.sign(exact)
    assert abs(large - exact) < 2e-4 * abs(exact)
    # the remaining error is the periodic-box error: it shrinks as the box grows
    assert abs(large - exact) < 0.2 * abs(small - exact)


@pytest.mark.parametrize("sr,sz", [(1.0, 0.6), (0.6, 1.0)])
def test_gaussian_dipolar_energy_anisotropic_grid(orc, sr, sz):
    """The closed form on a grid with unequal N and h per axis: 64 x 80 x 48 points at
    h = (0.3, 0.25, 0.4) (box 19.2 x 20 x 19.2), and the half-size grid (box halved)."""
    exact = e_dd_closed(sr, sz)
    h = (0.3, 0.25, 0.4)
    small = grid_e_dd(orc, (32, 40, 24), h, sr, sz)
    large = grid_e_dd(orc, (64, 80, 48), h, sr, sz)
    assert abs(large - exact) < 2e-4 * abs(exact)
    assert abs(large - exact) < 0.2 * abs(small - exact)


def test_isotropic_density_has_no_dipolar_energy(orc):
    assert abs(grid_e_dd(orc, 32, 0.3, 1.0, 1.0)) < 1e-15


@pytest.mark.parametrize("x", [1e-3, 0.1, 0.49, 0.5, 0.51, 1.0, 3.7, 12.0, 40.0])
def test_cutoff_factor_is_the_j2_integral(orc, x):
    """Spherical cutoff (interaction restricted to r < R): the kernel factor is
    3 int_0^{kR} j_2(t)/t dt (partial-wave expansion of the truncated 1/r^3 kernel),
    computed here by quadrature of the spherical Bessel function."""
    from scipy.special import spherical_jn
    val, _ = integrate.quad(lambda t: spherical_jn(2, t) / t, 0, x, limit=400, epsabs=1e-15, epsrel=1e-13)
    assert orc.cutoff_factor(x) == pytest.approx(3 * val, rel=1e-10, abs=1e-16)


def test_cutoff_tends_to_the_uncut_kernel(orc):
    # a cutoff much larger than the box changes only the lowest wavenumbers; R -> 0 removes
    # the interaction
    p0 = orc.make_params((8, 8, 8), 0.5, 1e-3, orc.REAL_TIME, (1, 1, 1), 0, 1)
    big = orc.make_params((8, 8, 8), 0.5, 1e-3, orc.REAL_TIME, (1, 1, 1), 0, 1, cutoff=1e4)
    tiny = orc.make_params((8, 8, 8), 0.5, 1e-3, orc.REAL_TIME, (1, 1, 1), 0, 1, cutoff=1e-6)
    u0, ub, ut = orc.dipolar_kernel(p0), orc.dipolar_kernel(big), orc.dipolar_kernel(tiny)
    assert np.max(np.abs(ub - u0)) < 1e-6
    assert np.max(np.abs(ut)) < 1e-11
