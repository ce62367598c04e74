"""Pins of the optional quadrature and derivative rules of the observables (the older
programs' Simpson rule and higher-order gradient): Simpson's weights integrate cubics
exactly, the rectangle rule does not; the 4th-order gradient's kinetic energy of the
harmonic-oscillator Gaussian converges as h^4 (the 3-point Laplacian's as h^2)."""
import numpy as np
import pytest

from paper_1610_05329_gb300 import inputs


def test_simpson_integrates_cubics_exactly(orc):
    n, h = (10, 12, 16), (0.3, 0.25, 0.2)
    x, y, z = inputs.grid_axes(n, h)
    # |psi|^2 = (x - x0)^3 (y - y0)^2 (z - z0 + 1), cubic in each coordinate, >= 0 on the grid
    f = ((x[:, None, None] - x[0]) ** 3) * ((y[None, :, None] - y[0]) ** 2) * (z[None, None, :] - z[0] + 1.0)
    psi = np.sqrt(f).astype(np.complex128)
    # exact integral over [x0, x_{n-2}] x [y0, y_{n-2}] x [z0, z_{n-2}]
    lx, ly, lz = (n[0] - 2) * h[0], (n[1] - 2) * h[1], (n[2] - 2) * h[2]
    exact = (lx ** 4 / 4) * (ly ** 3 / 3) * (lz ** 2 / 2 + lz)
    p_simp = orc.make_params(n, h, 1e-3, orc.REAL_TIME, (1, 1, 1), 0, 0, integration=1)
    p_rect = orc.make_params(n, h, 1e-3, orc.REAL_TIME, (1, 1, 1), 0, 0, integration=0)
    # the rectangle rule sums the last (wall) plane too: restrict that field to the same box
    assert orc.norm(p_simp, psi) == pytest.approx(exact, rel=1e-13)
    inner = psi.copy()
    inner[-1, :, :] = 0
    inner[:, -1, :] = 0
    inner[:, :, -1] = 0
    assert abs(orc.norm(p_rect, inner) - exact) > 1e-3 * exact


@pytest.mark.parametrize("kinetic,order", [(0, 2), (1, 4)])
def test_kinetic_energy_order(orc, kinetic, order):
    nu = (1.0, 1.5, 2.0)
    exact = sum(nu) / 4      # <p^2>/2 of the harmonic ground state
    errs = []
    for n, h in [(24, 0.5), (48, 0.25)]:
        x, y, z = inputs.grid_axes((n, n, n), h)
        psi = np.exp(-(nu[0] * x[:, None, None] ** 2 + nu[1] * y[None, :, None] ** 2
                       + nu[2] * z[None, None, :] ** 2) / 2).astype(np.complex128)
        p = orc.make_params((n, n, n), h, 1e-3, orc.IMAG_TIME, nu, 0, 0, kinetic=kinetic)
        psi /= np.sqrt(orc.norm(p, psi))
        errs.append(orc.observables(p, psi)["e_kin"] - exact)
    assert 0.8 * 2 ** order < errs[0] / errs[1] < 1.25 * 2 ** order
