"""Physics pins of the oracle's full SSCN step (potential, CN x/y/z, renormalisation).

The paper's programs find stationary states by propagating in imaginary time and follow
the dynamics by propagating in real time (Abstract; Solution method).  What the mathematics fixes:
  * non-interacting imaginary time converges to the harmonic ground state,
    mu = (nu_x + nu_y + nu_z)/2 and rms_d = 1/sqrt(2 nu_d), with O(h^2) grid error;
  * real time conserves the norm and is exactly reversible (dt -> -dt, reversed order);
  * a converged stationary state keeps its density under real time (to O(dt)) and its
    phase turns at the rate mu (which pins the step's theta against the mu formula);
  * the virial identity 2 E_kin - 2 E_trap + 3 (E_contact + E_dipolar) = 0 of the ground
    state (dilation argument), to the grid and splitting error;
  * Kohn's theorem: the centre of mass of a displaced ground state oscillates as
    x0 cos(nu_x t) whatever g and gdd are.
"""
import numpy as np
import pytest

from paper_1610_05329_gb300 import inputs


def ground_state(orc, n, h, dt, nu, g, gdd, tau):
    p = orc.make_params((n, n, n), h, dt, orc.IMAG_TIME, nu, g, gdd)
    psi = inputs.gaussian_psi((n, n, n), h, noise=0)
    return orc.step(p, psi, int(round(tau / dt))), p


def test_noninteracting_ground_state(orc):
    nu = (1.0, 1.5, 2.0)
    exact = sum(nu) / 2
    err = {}
    for n, h in [(24, 0.4), (48, 0.2)]:          # same box, +-4.8
        psi, p = ground_state(orc, n, h, 0.01, nu, 0.0, 0.0, 5.0)
        o = orc.observables(p, psi)
        assert o["norm"] == pytest.approx(1.0, abs=1e-12)
        err[h] = o["mu"] - exact
        if h == 0.2:
            for d in range(3):
                assert o["rms"][d] == pytest.approx(1 / np.sqrt(2 * nu[d]), rel=2e-4)
    assert abs(err[0.2]) < 0.012
    assert 3.6 < err[0.4] / err[0.2] < 4.4        # second-order 3-point Laplacian


def test_real_time_conserves_norm(orc):
    shape = (16, 12, 20)
    p = orc.make_params(shape, 0.4, 0.01, orc.REAL_TIME, (1.0, 0.8, 1.3), 30.0, 20.0)
    psi = inputs.gaussian_psi(shape, 0.4, seed=9)
    n0 = orc.observables(p, orc.cn_sweep(p, orc.cn_sweep(p, orc.cn_sweep(p, psi, 0), 1), 2))["norm"]
    out = orc.step(p, psi, 50)
    assert abs(orc.observables(p, out)["norm"] - n0) < 1e-13


def test_real_time_is_reversible(orc):
    shape = (12, 16, 10)
    p = orc.make_params(shape, 0.5, 0.02, orc.REAL_TIME, (1.0, 1.2, 0.9), 25.0, 15.0)
    back = orc.make_params(shape, 0.5, -0.02, orc.REAL_TIME, (1.0, 1.2, 0.9), 25.0, 15.0)
    psi = inputs.gaussian_psi(shape, 0.5, seed=2)
    for axis in range(3):      # a state of the Dirichlet box: zero on the walls
        psi[(slice(None),) * axis + (0,)] = 0
        psi[(slice(None),) * axis + (-1,)] = 0
    fwd = orc.step(p, psi, 10)
    rev = fwd
    for _ in range(10):   # inverse of (P, X, Y, Z) is (Z^-1, Y^-1, X^-1, P^-1)
        for axis in (2, 1, 0):
            rev = orc.cn_sweep(back, rev, axis)
        rev = orc.potential_step(back, rev)
    assert np.linalg.norm(rev - psi) < 1e-12 * np.linalg.norm(psi)
    assert np.linalg.norm(fwd - psi) > 1e-2 * np.linalg.norm(psi)


def test_stationary_state_and_phase_rate(orc):
    nu, g, gdd, n, h, t_end = (1.0, 1.0, 1.0), 10.0, 6.0, 24, 0.4, 0.4
    res = {}
    for dt in (0.01, 0.005):
        psi, p = ground_state(orc, n, h, dt, nu, g, gdd, 6.0)
        mu = orc.observables(p, psi)["mu"]
        pr = orc.make_params((n, n, n), h, dt, orc.REAL_TIME, nu, g, gdd)
        out = orc.step(pr, psi, int(round(t_end / dt)))
        dn = np.max(np.abs(np.abs(out) ** 2 - np.abs(psi) ** 2)) / np.max(np.abs(psi) ** 2)
        rate = -np.angle(np.vdot(psi, out)) / t_end
        res[dt] = (dn, rate - mu)
    # density change and phase-rate offset are first order in dt ...
    assert 1.8 < res[0.01][0] / res[0.005][0] < 2.2
    assert res[0.01][0] < 5e-3
    # ... and the extrapolated phase rate is mu (the dipolar part of mu alone is ~2e-2)
    assert abs(2 * res[0.005][1] - res[0.01][1]) < 2e-5


def test_virial_identity(orc):
    psi, p = ground_state(orc, 32, 0.3, 0.005, (1.0, 1.0, 1.0), 10.0, 6.0, 6.0)
    o = orc.observables(p, psi)
    virial = 2 * o["e_kin"] - 2 * o["e_trap"] + 3 * o["e_contact"] + 3 * o["e_dipolar"]
    assert o["e_contact"] > 0.3 * o["e_kin"]
    assert abs(virial) < 0.02 * o["e_kin"]


def test_kohn_dipole_mode(orc):
    nu, g, gdd, n, h = (1.3, 1.0, 1.2), 8.0, 5.0, 32, 0.3
    psi, p = ground_state(orc, n, h, 0.01, nu, g, gdd, 5.0)
    shift = 2
    moved = np.zeros_like(psi)
    moved[shift:] = psi[:-shift]
    x0 = shift * h
    x = (np.arange(n) - n // 2) * h

    def mean_x(f):
        d = np.abs(f) ** 2
        return np.sum(d * x[:, None, None]) / np.sum(d)

    base = mean_x(psi)
    dt = 0.005
    pr = orc.make_params((n, n, n), h, dt, orc.REAL_TIME, nu, g, gdd)
    chunk = int(round(np.pi / nu[0] / dt / 12))
    worst = 0.0
    f = moved
    for k in range(1, 13):
        f = orc.step(pr, f, chunk)
        t = k * chunk * dt
        worst = max(worst, abs(mean_x(f) - base - x0 * np.cos(nu[0] * t)))
    assert worst < 0.04 * x0
