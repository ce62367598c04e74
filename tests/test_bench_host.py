"""Host-side pieces of bench.py that need no GPU: the algorithmic flop counts behind the
FP64 roofline, the tracked physics of the timed steps, and the kernel-source key of the
stored ncu traffic."""
import math

import pytest

import bench


def test_flop_counts_of_the_256cubed_fp64_step():
    shape = (256, 256, 256)
    half = 129 / 256
    f = lambda k: bench.fp64_flops_per_point(k, shape, "fp64")
    # FFT of length n: 5 n log2 n per complex line; two real lines per complex z transform
    assert f("k1_density_r2c_z") == pytest.approx(2.5 * 8 + 5)
    assert f("k2_fft_y") == pytest.approx(5 * 8 * half)
    assert f("k4_ifft_y") == f("k2_fft_y")
    assert f("k3_fft_x_dipolar_ifft_x") == pytest.approx((10 * 8 + 2) * half)
    # per-line Crank-Nicolson: forward 8, backward 10, 2 chi - psi 4; K7 adds the sums
    assert f("k6_cn_y") == 22
    assert f("k7_cn_x_reduce") == 28
    # K5: C2R, unpacking, theta, sine/cosine (|theta| <= 1/8), rotation, the z sweep
    assert f("k5_c2r_z_phase_cn_z") == pytest.approx(2.5 * 8 + 2 + 9 + 18 + 6 + 22)
    assert f("not_a_kernel") == 0.0


def test_double_float_recovers_psi_and_fp32_sweeps_are_chunked():
    shape = (256, 256, 256)
    assert bench.fp64_flops_per_point("k6_cn_y", shape, "df64") == 30
    z_fp64 = bench.fp64_flops_per_point("k5_c2r_z_phase_cn_z", shape, "fp64")
    z_df64 = bench.fp64_flops_per_point("k5_c2r_z_phase_cn_z", shape, "df64")
    z_mixed = bench.fp64_flops_per_point("k5_c2r_z_phase_cn_z", shape, "mixed")
    assert z_df64 - z_fp64 == 8
    # the chunked solver: 8 + 10 + 16 + 4 + 88 / chunk, chunk 8 for lines of 254 unknowns
    assert z_mixed - z_fp64 == pytest.approx(16 + 88 / 8)


def test_track_physics():
    o0 = {"norm": 1.0, "energy": 2.0, "mu": 3.0, "rms": (1.0, 2.0, 3.0)}
    o1 = {"norm": 1.0 + 1e-12, "energy": 2.5, "mu": 3.5, "rms": (1.5, 2.5, 3.5)}
    p = bench.track_physics(o0, o1, 200)
    assert p["steps"] == 200
    assert p["norm_drift"] == pytest.approx(1e-12)
    assert p["energy_start"] == 2.0 and p["energy_end"] == 2.5 and p["mu_end"] == 3.5
    assert p["rms_start"] == [1.0, 2.0, 3.0] and p["rms_end"] == [1.5, 2.5, 3.5]


def test_single_process_aggregate_and_traffic_key():
    value, ms = bench.aggregate_over_ranks(8.0, 16 * 1000)
    assert ms == 8.0 and value == pytest.approx(16 * 1000 / 8e-3)
    key = bench.kernel_source_sha1()
    assert len(key) == 40 and all(ch in "0123456789abcdef" for ch in key)
    # every stored traffic figure is a positive byte count of a known workload's K5
    for sha, table in bench.NCU_TRAFFIC.items():
        for (workload, kernel), nbytes in table.items():
            assert workload in bench.WORKLOADS and kernel == "k5_c2r_z_phase_cn_z"
            assert nbytes > 0 and math.isfinite(nbytes)


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference (the oracle on the host cores) prints one JSON line with the
    reference keys; one full 256^3 step after three warm-up steps."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 3
    assert line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
