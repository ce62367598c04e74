"""Pins of the oracle's discrete adjoint of the real-time SSCN step (the differentiation
workload: gradients of <z^2> of the final state w.r.t. a piecewise-constant nu_z schedule,
g and gdd).  The adjoint is pinned against the oracle's own forward step, which the other
oracle tests pin against the physics:
  * dot-product test <w, J v> = <J^T w, v> with J v by central differences;
  * parameter derivatives of a linear functional of one step by central differences;
  * the whole schedule gradient by central differences (h = 1e-6, FP64)."""
import numpy as np
import pytest

from paper_1610_05329_gb300 import inputs

SHAPE, H = (12, 10, 14), 0.55


def params(orc, dt=0.01, g=30.0, gdd=18.0, nu=(1.0, 1.2, 0.9)):
    return orc.make_params(SHAPE, H, dt, orc.REAL_TIME, nu, g, gdd)


def re_dot(a, b):
    return float(np.real(np.vdot(a, b)))


def walled(psi):
    psi = psi.copy()
    for axis in range(3):
        psi[(slice(None),) * axis + (0,)] = 0
        psi[(slice(None),) * axis + (-1,)] = 0
    return psi


def test_dot_product_identity(orc):
    p = params(orc)
    psi = walled(inputs.gaussian_psi(SHAPE, H, seed=4))
    v = walled(inputs.random_psi(SHAPE, seed=8, scale=0.1))
    w = inputs.random_psi(SHAPE, seed=9)
    eps = 1e-6
    jv = (orc.step(p, psi + eps * v) - orc.step(p, psi - eps * v)) / (2 * eps)
    jtw, _ = orc.adjoint_step(p, psi, w)
    lhs, rhs = re_dot(w, jv), re_dot(jtw, v)
    assert abs(lhs - rhs) < 1e-7 * max(abs(lhs), 1e-3)


@pytest.mark.parametrize("which", ["g", "gdd", "nu_z"])
def test_parameter_derivatives_of_one_step(orc, which):
    psi = walled(inputs.gaussian_psi(SHAPE, H, seed=5))
    w = inputs.random_psi(SHAPE, seed=11)
    base = dict(g=30.0, gdd=18.0, nu=(1.0, 1.2, 0.9))

    def loss(delta):
        kw = dict(base)
        if which == "nu_z":
            kw["nu"] = (1.0, 1.2, 0.9 + delta)
        else:
            kw[which] = base[which] + delta
        return re_dot(w, orc.step(params(orc, **kw), psi))

    eps = 1e-6
    fd = (loss(eps) - loss(-eps)) / (2 * eps)
    _, grads = orc.adjoint_step(params(orc), psi, w)
    got = grads[{"g": 0, "gdd": 1, "nu_z": 2}[which]]
    assert abs(got - fd) < 1e-6 * max(abs(fd), 1e-6)


def test_schedule_gradient_by_central_differences(orc):
    p = params(orc, dt=0.02)
    psi0 = inputs.gaussian_psi(SHAPE, H, seed=6, center=(0.2, -0.1, 0.3))
    nu_z = np.array([0.9, 1.15, 1.05])
    spb = 4
    loss, dnu, dg, dgdd = orc.grad_z2(p, nu_z, spb, psi0)
    eps = 1e-6

    def l_of(nu=nu_z, g=30.0, gdd=18.0):
        q = orc.make_params(SHAPE, H, 0.02, orc.REAL_TIME, (1.0, 1.2, 0.9), g, gdd)
        return orc.grad_z2(q, nu, spb, psi0)[0]

    for s in range(nu_z.size):
        up, dn = nu_z.copy(), nu_z.copy()
        up[s] += eps
        dn[s] -= eps
        fd = (l_of(nu=up) - l_of(nu=dn)) / (2 * eps)
        assert abs(dnu[s] - fd) < 1e-6 * max(abs(fd), 1e-4), (s, dnu[s], fd)
    fd_g = (l_of(g=30.0 + eps) - l_of(g=30.0 - eps)) / (2 * eps)
    fd_gdd = (l_of(gdd=18.0 + eps) - l_of(gdd=18.0 - eps)) / (2 * eps)
    assert abs(dg - fd_g) < 1e-6 * max(abs(fd_g), 1e-6)
    assert abs(dgdd - fd_gdd) < 1e-6 * max(abs(fd_gdd), 1e-6)
    assert loss > 0
