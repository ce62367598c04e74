"""Batched condensates (one CUDA graph, one branch per condensate) and the launch-shape
autotuner: batching must not change any result (bitwise), tuning must leave the state
untouched and the results within the parity tolerance of the oracle."""
import numpy as np
import pytest

from paper_1610_05329_gb300 import abi, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1610_05329_gb300 import build
    build.build()
    abi.load()


MEMBERS = [((16, 16, 16), 0.6, abi.DGPE_IMAG_TIME, (1.0, 1.3, 0.7), 12.0, 6.0),
           ((24, 24, 24), 0.45, abi.DGPE_IMAG_TIME, (0.6, 1.0, 1.8), 60.0, 40.0),
           ((32, 18, 12), 0.5, abi.DGPE_REAL_TIME, (1.0, 1.0, 1.0), 30.0, 10.0),
           ((12, 48, 24), 0.35, abi.DGPE_REAL_TIME, (2.0, 0.5, 1.1), 5.0, 4.0)]


@pytest.mark.parametrize("precision", [abi.DGPE_FP64, abi.DGPE_MIXED, abi.DGPE_DF64])
def test_batch_equals_individual_steps(precision):
    cdt = np.complex64 if precision == abi.DGPE_MIXED else np.complex128
    batched, alone = [], []
    for k, (shape, h, mode, nu, g, gdd) in enumerate(MEMBERS):
        psi = inputs.gaussian_psi(shape, h, seed=20 + k).astype(cdt)
        for group in (batched, alone):
            c = abi.Condensate(shape, h, 0.005, mode=mode, precision=precision, nu=nu, g=g, gdd=gdd)
            c.set_psi(psi)
            group.append(c)
    b = abi.Batch(batched)
    b.step(7)
    b.sync()
    for c in alone:
        c.step(7)
    for x, y in zip(batched, alone):
        assert np.array_equal(x.get_psi(), y.get_psi())
    # a parameter change rebuilds the batch graph
    batched[0].set_params(g=20.0)
    alone[0].set_params(g=20.0)
    b.step(3)
    b.sync()
    alone[0].step(3)
    assert np.array_equal(batched[0].get_psi(), alone[0].get_psi())
    b.close()
    for c in batched + alone:
        c.close()


def test_autotune_restores_state_and_keeps_parity(orc):
    shape, h, dt = (32, 48, 24), 0.3, 0.005
    psi = inputs.gaussian_psi(shape, h, seed=31)
    c = abi.Condensate(shape, h, dt, mode=abi.DGPE_REAL_TIME, nu=(1.0, 1.1, 0.9), g=25.0, gdd=15.0)
    c.set_psi(psi)
    t = c.autotune()
    assert t["step_ms_tuned"] > 0 and t["step_ms_default"] > 0
    assert np.array_equal(c.get_psi(), psi)
    c.step(6)
    p = orc.make_params(shape, h, dt, orc.REAL_TIME, (1.0, 1.1, 0.9), 25.0, 15.0)
    want = orc.step(p, psi, 6)
    got = c.get_psi()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-10
    # every radix order gives the same step within the FP64 parity bar
    for style in (0, 1, 2):
        c.set_tuning(dict(t, plan_style=(style, style, style)))
        c.set_psi(psi)
        c.step(6)
        assert np.linalg.norm(c.get_psi() - want) / np.linalg.norm(want) < 1e-10
    with pytest.raises(abi.DgpeError):
        c.set_tuning(dict(t, ylines=3))
    c.close()


def test_autotune_double_float(orc):
    """The autotuner and every radix order on the double-float path, against the oracle."""
    shape, h, dt = (32, 48, 24), 0.3, 0.005
    psi = inputs.gaussian_psi(shape, h, seed=33)
    c = abi.Condensate(shape, h, dt, mode=abi.DGPE_REAL_TIME, precision=abi.DGPE_DF64, nu=(1.0, 1.1, 0.9),
                       g=25.0, gdd=15.0)
    c.set_psi(psi)
    t = c.autotune()
    assert np.max(np.abs(c.get_psi() - psi)) < 2.0 ** -47 * np.max(np.abs(psi))
    p = orc.make_params(shape, h, dt, orc.REAL_TIME, (1.0, 1.1, 0.9), 25.0, 15.0)
    want = orc.step(p, psi, 6)
    for style in (0, 1, 2):
        c.set_tuning(dict(t, plan_style=(style, style, style)))
        c.set_psi(psi)
        c.step(6)
        assert np.linalg.norm(c.get_psi() - want) / np.linalg.norm(want) < 1e-10
    c.close()


def test_batch_step_counts_and_graph_cache():
    """dgpe_batch_step(b, n) runs each member's n steps as one chain in one graph launch;
    graphs are cached per step count (at most four).  Any sequence of calls, with more
    distinct counts than the cache holds, equals the members' own steps bitwise."""
    batched, alone = [], []
    for k, (shape, h, mode, nu, g, gdd) in enumerate(MEMBERS):
        psi = inputs.gaussian_psi(shape, h, seed=40 + k).astype(np.complex64)
        for group in (batched, alone):
            c = abi.Condensate(shape, h, 0.004, mode=mode, precision=abi.DGPE_MIXED, nu=nu, g=g, gdd=gdd)
            c.set_psi(psi)
            group.append(c)
    b = abi.Batch(batched)
    counts = [2, 5, 2, 1, 4, 3, 6, 5]
    for n in counts:
        b.step(n)
    b.sync()
    for c in alone:
        c.step(sum(counts))
    for x, y in zip(batched, alone):
        assert np.array_equal(x.get_psi(), y.get_psi())
    b.close()
    for c in batched + alone:
        c.close()


@pytest.mark.parametrize("mode", [abi.DGPE_IMAG_TIME, abi.DGPE_REAL_TIME])
# (the second: short-line sweeps; the last three: K5's compile-time z lengths with the 8-lane z solve)
@pytest.mark.parametrize("shape", [(24, 20, 32), (32, 48, 20), (20, 24, 64), (24, 20, 96), (16, 20, 128)])
def test_grouped_members_equal_individual_steps(mode, shape):
    """Same-shaped FP32 members (different physics and states) are stepped as one group, each
    kernel one launch for all of them; a member of another shape and an FP64 member run as
    branches of their own.  Every result equals the member's own steps bitwise, before and
    after a parameter change (which rebuilds the grouped launches' argument array)."""
    h = 0.45
    specs = [((1.0, 1.2, 0.8), 30.0, 10.0), ((0.7, 1.0, 1.5), 55.0, 40.0), ((1.3, 0.9, 1.1), 8.0, 2.0)]
    batched, alone = [], []
    for k, (nu, g, gdd) in enumerate(specs):
        psi = inputs.gaussian_psi(shape, h, seed=60 + k).astype(np.complex64)
        for group in (batched, alone):
            c = abi.Condensate(shape, h, 0.004, mode=mode, precision=abi.DGPE_MIXED, nu=nu, g=g, gdd=gdd)
            c.set_psi(psi)
            group.append(c)
    for k, (shp, prec) in enumerate([((16, 24, 20), abi.DGPE_MIXED), (shape, abi.DGPE_FP64)]):
        cdt = np.complex64 if prec == abi.DGPE_MIXED else np.complex128
        psi = inputs.gaussian_psi(shp, h, seed=70 + k).astype(cdt)
        for group in (batched, alone):
            c = abi.Condensate(shp, h, 0.004, mode=mode, precision=prec, nu=(1.0, 1.0, 1.0), g=20.0, gdd=5.0)
            c.set_psi(psi)
            group.append(c)
    b = abi.Batch(batched)
    b.step(6)
    b.sync()
    for c in alone:
        c.step(6)
    for x, y in zip(batched, alone):
        assert np.array_equal(x.get_psi(), y.get_psi())
    batched[1].set_params(g=12.0)
    alone[1].set_params(g=12.0)
    b.step(4)
    b.sync()
    for c in alone:
        c.step(4)
    for x, y in zip(batched, alone):
        assert np.array_equal(x.get_psi(), y.get_psi())
    b.close()
    for c in batched + alone:
        c.close()
