"""Pins of the oracle's Crank-Nicolson kinetic sweeps (Thomas algorithm).

The kinetic part of the split-step Crank-Nicolson method (paper, Solution method) is a
batch of tridiagonal solves.  Pins: Thomas equals a dense LU solve; each sweep equals the
dense Cayley map (I - cD)^{-1}(I + cD) on the interior of every line (Dirichlet walls);
the real-time sweep is unitary; sweeps along different axes commute (tensor-product
operators), which is what lets the GPU run them in another order.
"""
import numpy as np
import pytest

from paper_1610_05329_gb300 import inputs


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("n", list(range(1, 17)))
def test_thomas_equals_dense_solve(orc, n):
    lo = inputs.random_psi((n,), seed=n)
    up = inputs.random_psi((n,), seed=n + 50)
    di = 3.0 + inputs.random_psi((n,), seed=n + 99)   # diagonally dominant
    rhs = inputs.random_psi((n,), seed=n + 7)
    a = np.diag(di) + np.diag(lo[1:], -1) + np.diag(up[:-1], 1)
    x = orc.thomas(lo, di, up, rhs)
    assert rel(x, np.linalg.solve(a, rhs)) < 1e-14
    assert np.linalg.norm(a @ x - rhs) < 1e-14 * np.linalg.norm(rhs) * 10


def dense_cn_line(line, c):
    n = line.size
    m = n - 2
    d = np.diag(-2.0 * np.ones(m)) + np.diag(np.ones(m - 1), 1) + np.diag(np.ones(m - 1), -1)
    a = np.eye(m) - c * d
    b = np.eye(m) + c * d
    out = np.zeros_like(line)
    out[1:-1] = np.linalg.solve(a, b @ line[1:-1])
    return out


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sweep_equals_dense_cayley(orc, mode, axis):
    shape = (6, 8, 10)
    h = (0.3, 0.25, 0.2)
    dt = 0.05
    p = orc.make_params(shape, h, dt, mode, (1, 1, 1), 0, 0)
    psi = inputs.random_psi(shape, seed=21)
    out = orc.cn_sweep(p, psi, axis)
    r = dt / (4 * h[axis] ** 2)
    c = 1j * r if mode == orc.REAL_TIME else r
    want = np.apply_along_axis(lambda l: dense_cn_line(l, c), axis, psi)
    assert rel(out, want) < 1e-14


def test_real_time_sweep_is_unitary(orc):
    shape = (8, 12, 16)
    p = orc.make_params(shape, 0.2, 0.01, orc.REAL_TIME, (1, 1, 1), 0, 0)
    psi = inputs.random_psi(shape, seed=3)
    for axis in range(3):
        psi[(slice(None),) * axis + (0,)] = 0
        psi[(slice(None),) * axis + (-1,)] = 0
    n0 = np.vdot(psi, psi).real
    for axis in range(3):
        psi = orc.cn_sweep(p, psi, axis)
        assert abs(np.vdot(psi, psi).real - n0) < 1e-13 * n0


@pytest.mark.parametrize("mode", [0, 1])
def test_sweeps_commute(orc, mode):
    shape = (8, 12, 10)
    p = orc.make_params(shape, (0.3, 0.2, 0.25), 0.02, mode, (1, 1, 1), 0, 0)
    psi = inputs.random_psi(shape, seed=4)
    a = psi
    for axis in (0, 1, 2):
        a = orc.cn_sweep(p, a, axis)
    b = psi
    for axis in (2, 1, 0):
        b = orc.cn_sweep(p, b, axis)
    assert rel(a, b) < 1e-14
    assert rel(a, psi) > 1e-3   # the sweeps did something
