"""Stored fixtures under tests/golden/.

* paper_3d_timings.txt: the paper's only printed numbers, the wall-clock times of its 3D
  programs (Tables 1-3).  bench.py quotes them beside its own times on the same grids; this
  checks that every quoted figure is the paper's and that the grids match.
* oracle_imag64.txt: the FP64 oracle's observables after the 64^3 imaginary-time workload,
  written by tests/golden/make_oracle_golden.py (oracle and seeded inputs only).  The oracle
  must reproduce it (a regression guard, not an independent pin), and the GPU FP64 path must
  match it at the parity bar.
"""
import os
import re

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def paper_rows():
    rows = []
    for line in open(os.path.join(GOLDEN, "paper_3d_timings.txt")):
        if line.startswith("#") or not line.strip():
            continue
        prog, grid, conf, sec = line.split()
        rows.append((prog, grid, conf, int(sec)))
    return rows


def oracle_golden():
    vals = {}
    for line in open(os.path.join(GOLDEN, "oracle_imag64.txt")):
        if not line.startswith("#") and line.strip():
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_bench_quotes_the_paper_tables():
    import bench
    rows = paper_rows()
    assert len(rows) == 10
    for grid, item in bench.PAPER_GRIDS.items():
        assert tuple(item["shape"]) == tuple(int(x) for x in grid.split("x"))
        quoted = {int(x) for x in re.findall(r"\d+", item["paper"])}
        want = {sec for _, g, _, sec in rows if g == grid}
        assert want and want <= quoted, grid


def test_paper_rates_from_the_tables():
    """The grid-point update rates behind the paper's rows (N_tot x 1000 / seconds), e.g.
    480^3 x 1000 / 888 s = 1.245e8 updates/s for imag3d-th."""
    rates = {}
    for prog, grid, conf, sec in paper_rows():
        n = 1
        for x in grid.split("x"):
            n *= int(x)
        rates[(prog, conf)] = n * 1000 / sec
    assert rates[("imag3d-th", "T=16")] == pytest.approx(1.2454e8, rel=1e-4)
    assert rates[("real3d-mpicuda", "N=1")] == pytest.approx(480 * 480 * 250 * 1000 / 800)
    # the fastest 3D figure the paper prints: 32 nodes of 16 cores, imaginary time, 1.2e9
    assert max(rates.values()) == rates[("imag3d-mpi", "N=32")]
    assert rates[("imag3d-mpi", "N=32")] == pytest.approx(1.2e9)


def test_oracle_reproduces_its_golden_fixture():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_oracle_golden", os.path.join(GOLDEN, "make_oracle_golden.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    got, want = gen.compute(), oracle_golden()
    for k, v in want.items():
        # another host compiler may contract multiply-adds differently: 1e-10, not bit equality
        assert got[k] == pytest.approx(v, rel=1e-10, abs=1e-12), k


@pytest.mark.gpu
def test_gpu_fp64_matches_the_oracle_golden_fixture():
    import torch
    from paper_1610_05329_gb300 import abi, build, inputs
    build.build()
    assert torch.cuda.is_available()
    shape, h = (64, 64, 64), 0.2
    gpu = abi.Condensate(shape, h, 0.004, mode=abi.DGPE_IMAG_TIME, precision=abi.DGPE_FP64, nu=(1.0, 1.0, 1.0),
                         g=20.0, gdd=10.0)
    gpu.set_psi(inputs.gaussian_psi(shape, h, noise=1e-3, seed=1))
    gpu.step(200)
    obs = gpu.observables()
    gpu.close()
    obs["rms_x"], obs["rms_y"], obs["rms_z"] = obs.pop("rms")
    for k, v in oracle_golden().items():
        assert obs[k] == pytest.approx(v, rel=1e-10, abs=1e-12), k
