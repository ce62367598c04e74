#!/usr/bin/env python3
"""Throughput of the 3D dipolar GP split-step Crank-Nicolson step on GB300.

Default workload (N=1): the real-time FP64 step on a 256^3 grid (h = 0.1, trap
(0.5, 1.0, 1.5), gdd = 25, quench g 50 -> 40, dt = 5e-4).  The state is the seeded
Gaussian (width 1, 1e-3 noise, seed 1) after 20 imaginary-time steps at g = 50 (a short
preparation, not a converged ground state: the cost of a step does not depend on the
state).  Metric: grid-point updates per second, nx*ny*nz*steps / time.  psi (268 MB) is
larger than the 129 MB L2, so no flush is needed between steps.

The same JSON line also carries the FP32-mixed step on 512x512x384 (h = 0.05, trap
(1, 1, 2), g = 100, gdd = 60, real time dt = 5e-4) as "mixed_512x512x384".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the workload on its own
GPU (the single-grid step is not sharded); value = all ranks' updates / max rank time.
--impl reference times the FP64 CPU oracle on the host cores (rank 0 only).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3D SSCN grid-point updates/s (256^3 FP64 real time)"
UNIT = "grid-point updates/s"

WORKLOADS = {
    "real256_fp64": dict(shape=(256, 256, 256), h=0.1, nu=(0.5, 1.0, 1.5), g_prep=50.0, g=40.0, gdd=25.0,
                         dt_prep=0.004, dt=5e-4, precision="fp64"),
    "real512x512x384_mixed": dict(shape=(512, 512, 384), h=0.05, nu=(1.0, 1.0, 2.0), g_prep=100.0, g=100.0,
                                  gdd=60.0, dt_prep=0.001, dt=5e-4, precision="mixed"),
    # the 256^3 workload in double-float (FP32 pairs on the FP32 pipe)
    "real256_df64": dict(shape=(256, 256, 256), h=0.1, nu=(0.5, 1.0, 1.5), g_prep=50.0, g=40.0, gdd=25.0,
                         dt_prep=0.004, dt=5e-4, precision="df64"),
}
PRECISIONS = {"fp64": 0, "mixed": 1, "df64": 2}   # DGPE_FP64, DGPE_MIXED, DGPE_DF64
PREP_STEPS = 20

# FP64 peak of GB300 from its unit counts and clock: 152 SMs x 2 FP64 FMA per clock per SM
# (measured issue rate) x 2 flops x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12

# DRAM bytes (read + write) per launch from ncu captures (profiles/), valid while the kernel
# source is byte-identical to the one captured (sha1 of dgpe_device.cuh).
NCU_TRAFFIC = {
    # FP64 and double-float: the K5 record times two launches (the phase-only pass and the
    # two-thread z sweep)
    "c2daf7f0f7773df816b53dbc0e6220ab5d8756a2": {
        ("real256_fp64", "k5_c2r_z_phase_cn_z"): 1850.61e6,
        ("real512x512x384_mixed", "k5_c2r_z_phase_cn_z"): 1961.65e6,
    },
}


def kernel_source_sha1():
    import hashlib
    path = os.path.join(ROOT, "paper_1610_05329_gb300", "csrc", "dgpe_device.cuh")
    with open(path, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()


def fp64_flops_per_point(kernel, shape, precision="fp64"):
    """Algorithmic FP64 flops per grid point of each real-time kernel (FMA = 2 flops) as the
    kernels compute them; the derivation is in the design notes.  FFT of length n: 5 n log2 n
    per complex line; the half spectrum has (nz/2+1)/nz complex values per real point.
    Crank-Nicolson: the chunked warp solver (forward, backward, chunk fix-up, 2chi - psi,
    lane scans) or the one-thread-per-line Thomas solver (forward, backward, 2chi - psi; in
    double-float also psi recovered from y, which FP64 reads back instead)."""
    import math
    nx, ny, nz = shape
    half = (nz // 2 + 1) / nz
    chunk = 2
    while chunk * 32 < nz - 2:
        chunk *= 2
    cn_chunked = 8 + 10 + 16 + 4 + 88.0 / chunk
    cn_line = 8 + 10 + 4 + (8 if precision == "df64" else 0)
    # FP64 and double-float: every sweep per line (two threads each); FP32: chunked
    cn_z = cn_line if precision in ("fp64", "df64") else cn_chunked
    return {
        "k1_density_r2c_z": 2.5 * math.log2(nz) + 5,
        "k2_fft_y": 5 * math.log2(ny) * half,
        "k3_fft_x_dipolar_ifft_x": (10 * math.log2(nx) + 2) * half,
        "k4_ifft_y": 5 * math.log2(ny) * half,
        # sine/cosine: 18 flops for |theta| <= 1/8 (99.5 % of this workload's points; the
        # rest up to 0.15), 22 up to 1/4, else 36 + reduction
        "k5_c2r_z_phase_cn_z": 2.5 * math.log2(nz) + 2 + 9 + 18 + 6 + cn_z,
        "k6_cn_y": cn_line,
        "k7_cn_x_reduce": cn_line + 6,
    }.get(kernel, 0.0)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[4], f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[3:]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def make_condensate(abi, wl, local):
    import torch
    from paper_1610_05329_gb300 import inputs
    prec = PRECISIONS[wl["precision"]]
    c = abi.Condensate(wl["shape"], wl["h"], wl["dt_prep"], mode=abi.DGPE_IMAG_TIME, precision=prec,
                       nu=wl["nu"], g=wl["g_prep"], gdd=wl["gdd"], device=torch.device("cuda", local))
    psi0 = inputs.gaussian_psi(wl["shape"], wl["h"], noise=1e-3, seed=1)
    c.set_psi(torch.from_numpy(psi0).to(device=c.device, dtype=c.cdtype))
    c.step(PREP_STEPS)
    c.set_params(mode=abi.DGPE_REAL_TIME, dt=wl["dt"], g=wl["g"])
    return c


def aggregate_over_ranks(ms_local, units_per_rank, dist=None, device=None):
    """Whole-job throughput of independent replicas: every rank processed units_per_rank
    units; the job time is the slowest rank's (MAX all-reduce).  Returns (value, ms)."""
    ms = float(ms_local)
    ws = 1
    if dist is not None and dist.is_initialized():
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        ws = dist.get_world_size()
    return ws * units_per_rank / (ms * 1e-3), ms


def track_physics(obs0, obs1, steps):
    """Norm drift, energy and rms sizes over the timed real-time steps (the quantities the
    workload tracks)."""
    return {"steps": steps, "norm_start": obs0["norm"], "norm_end": obs1["norm"],
            "norm_drift": (obs1["norm"] - obs0["norm"]) / obs0["norm"],
            "energy_start": obs0["energy"], "energy_end": obs1["energy"], "mu_end": obs1["mu"],
            "rms_start": list(obs0["rms"]), "rms_end": list(obs1["rms"])}


# The mixed-precision workload as defined: 512x512x384, h = 0.05, trap (1, 1, 2), g = 100,
# gdd = 60; imaginary time at dt = 0.001, then real time at dt = 5e-4 (the unstated steps).
PRECISION_WL = dict(shape=(512, 512, 384), h=0.05, nu=(1.0, 1.0, 2.0), g=100.0, gdd=60.0, dt_imag=0.001,
                    dt_real=5e-4)
MIXED_DTYPE = "f32 (reductions: FP32 terms, exact weights, double-float sums per point, FP64 across blocks)"


def rel_errors(psi, obs, psi_ref, obs_ref):
    """Errors of (psi, obs) against a reference: rel-L2 of psi and the relative errors of
    mu, E, the rms sizes and the norm."""
    import torch
    # the same after removing the best global phase e^{i phi}, phi = arg <psi_ref, psi>
    ov = torch.vdot(psi_ref.flatten(), psi.flatten())
    aligned = psi * (ov.conj() / abs(ov)) if abs(ov) > 0 else psi
    return {"psi_rel_l2": float(torch.linalg.norm(psi - psi_ref) / torch.linalg.norm(psi_ref)),
            "psi_rel_l2_phase_aligned": float(torch.linalg.norm(aligned - psi_ref) / torch.linalg.norm(psi_ref)),
            "mu_rel": abs(obs["mu"] - obs_ref["mu"]) / abs(obs_ref["mu"]),
            "energy_rel": abs(obs["energy"] - obs_ref["energy"]) / abs(obs_ref["energy"]),
            "rms_rel": [abs(a - b) / abs(b) for a, b in zip(obs["rms"], obs_ref["rms"])],
            "norm_rel": abs(obs["norm"] - obs_ref["norm"]) / abs(obs_ref["norm"])}


def run_phases(abi, local, precision, imag_steps, real_steps):
    """The mixed-precision workload from the seeded Gaussian (width 1, 1e-3 noise, seed 1):
    `imag_steps` imaginary-time steps, then `real_steps` real-time steps; the observables and
    psi (complex128, on the device) after each phase."""
    import torch
    from paper_1610_05329_gb300 import inputs
    wl = PRECISION_WL
    c = abi.Condensate(wl["shape"], wl["h"], wl["dt_imag"], mode=abi.DGPE_IMAG_TIME, precision=PRECISIONS[precision],
                       nu=wl["nu"], g=wl["g"], gdd=wl["gdd"], device=torch.device("cuda", local))
    psi0 = inputs.gaussian_psi(wl["shape"], wl["h"], noise=1e-3, seed=1)
    c.set_psi(torch.from_numpy(psi0).to(device=c.device, dtype=c.cdtype))
    c.step(imag_steps)
    out = [(c.observables(), c.get_psi(host=False).to(torch.complex128))]
    c.set_params(mode=abi.DGPE_REAL_TIME, dt=wl["dt_real"])
    c.step(real_steps)
    out.append((c.observables(), c.get_psi(host=False).to(torch.complex128)))
    c.close()
    return out


def precision_table(abi, local, imag_steps=500, real_steps=500):
    """Error table of the FP32-mixed path on its workload against the FP64 GPU path, after
    `imag_steps` imaginary-time and then `real_steps` real-time steps, each path from the same
    seeded state.  (The comparison of both paths with the FP64 oracle at this size, over the
    few steps the host cores finish in seconds, is a GPU test.)"""
    import torch
    wl = PRECISION_WL
    t0 = time.perf_counter()
    mixed = run_phases(abi, local, "mixed", imag_steps, real_steps)
    fp64 = run_phases(abi, local, "fp64", imag_steps, real_steps)
    table = {"grid": list(wl["shape"]), "h": wl["h"], "nu": list(wl["nu"]), "g": wl["g"], "gdd": wl["gdd"],
             "dt_imag": wl["dt_imag"], "dt_real": wl["dt_real"], "start": "seeded Gaussian (width 1, 1e-3 noise, seed 1)",
             "vs_fp64_gpu": {"after_imag": dict(steps=imag_steps, **rel_errors(*mixed[0][::-1], *fp64[0][::-1])),
                             "after_real": dict(steps=real_steps, **rel_errors(*mixed[1][::-1], *fp64[1][::-1])),
                             "fp64_after_imag": {k: fp64[0][0][k] for k in ("mu", "energy", "rms", "norm")},
                             "fp64_after_real": {k: fp64[1][0][k] for k in ("mu", "energy", "rms", "norm")}},
             "wall_s": None}
    del mixed, fp64
    torch.cuda.empty_cache()
    table["wall_s"] = round(time.perf_counter() - t0, 2)
    return table


def ground_state_run(abi, local, tol=1e-10, check_every=100, max_steps=20000, real_steps=1000, record_every=100):
    """The 256^3 real-time workload as defined: the imaginary-time ground state (FP64,
    dt = 0.004, g = 50) from the seeded Gaussian, run until mu changes by less than `tol`
    between checks `check_every` steps apart (at most `max_steps`); then the quench g -> 40
    and `real_steps` real-time steps at dt = 5e-4, with the norm, energy and rms sizes every
    `record_every` steps."""
    import torch
    from paper_1610_05329_gb300 import inputs
    wl = WORKLOADS["real256_fp64"]
    c = abi.Condensate(wl["shape"], wl["h"], wl["dt_prep"], mode=abi.DGPE_IMAG_TIME, precision=abi.DGPE_FP64,
                       nu=wl["nu"], g=wl["g_prep"], gdd=wl["gdd"], device=torch.device("cuda", local))
    c.set_psi(torch.from_numpy(inputs.gaussian_psi(wl["shape"], wl["h"], noise=1e-3, seed=1)).to(
        device=c.device, dtype=c.cdtype))
    t0 = time.perf_counter()
    steps, mu_prev, dmu = 0, None, None
    while steps < max_steps:
        c.step(check_every)
        steps += check_every
        mu = c.observables()["mu"]
        if mu_prev is not None:
            dmu = abs(mu - mu_prev)
            if dmu < tol:
                break
        mu_prev = mu
    gs = c.observables()
    imag_s = time.perf_counter() - t0
    c.set_params(mode=abi.DGPE_REAL_TIME, dt=wl["dt"], g=wl["g"])
    o0 = c.observables()
    series = [{"step": 0, "norm": o0["norm"], "energy": o0["energy"], "rms": list(o0["rms"])}]
    t1 = time.perf_counter()
    for k in range(real_steps // record_every):
        c.step(record_every)
        o = c.observables()
        series.append({"step": (k + 1) * record_every, "norm": o["norm"], "energy": o["energy"], "rms": list(o["rms"])})
    real_s = time.perf_counter() - t1
    c.close()
    n0 = series[0]["norm"]
    return {"grid": list(wl["shape"]), "imag": {"dt": wl["dt_prep"], "g": wl["g_prep"], "steps": steps,
                                                "converged": dmu is not None and dmu < tol,
                                                "criterion": "|delta mu| < %g between checks %d steps apart" % (tol, check_every),
                                                "final_delta_mu": dmu, "mu": gs["mu"], "energy": gs["energy"],
                                                "rms": list(gs["rms"]), "wall_s": round(imag_s, 2)},
            "real": {"dt": wl["dt"], "g": wl["g"], "steps": real_steps,
                     "norm_drift": (series[-1]["norm"] - n0) / n0,
                     "max_norm_deviation": max(abs(r["norm"] - n0) for r in series) / n0,
                     "energy_drift": (series[-1]["energy"] - series[0]["energy"]) / abs(series[0]["energy"]),
                     "series": series, "wall_s": round(real_s, 2)}}


def time_steps(c, steps, barrier):
    import torch
    st = c.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize(c.device)
    e0.record(st)
    c.step(steps)
    e1.record(st)
    torch.cuda.synchronize(c.device)
    barrier()
    return e0.elapsed_time(e1)


def kernel_profile(c, steps, hbm_peak, peak_kind, workload):
    """Per-kernel CUDA-event durations over `steps` instrumented steps (the same step
    sequence as the timed region, with an event pair around every launch)."""
    import torch
    wl = WORKLOADS[workload]
    npts = wl["shape"][0] * wl["shape"][1] * wl["shape"][2]
    c.set_timing(True)
    c.kernel_times()        # reset
    t0 = time.perf_counter()
    c.step(steps)
    torch.cuda.synchronize(c.device)
    wall = time.perf_counter() - t0
    rows = c.kernel_times()
    c.set_timing(False)
    total = sum(r["total_ms"] for r in rows)
    traffic = NCU_TRAFFIC.get(kernel_source_sha1(), {})
    out = []
    for r in rows:
        avg = r["total_ms"] / r["launches"]
        gbs = r["bytes_per_launch"] / (avg * 1e-3) / 1e9
        d = {"kernel": r["name"], "launches": r["launches"], "avg_ms": round(avg, 5),
             "share": round(r["total_ms"] / total, 4), "bytes_per_launch": r["bytes_per_launch"],
             "achieved_gbs": round(gbs, 1), "frac_hbm": round(gbs / hbm_peak, 4)}
        if wl["precision"] in ("fp64", "df64"):
            fl = fp64_flops_per_point(r["name"], wl["shape"], wl["precision"]) * npts
            d["fp64_flops_per_launch"] = fl
            d["fp64_tflops"] = round(fl / (avg * 1e-3) / 1e12, 4)
            d["frac_fp64"] = round(d["fp64_tflops"] / FP64_PEAK_TFLOPS, 4)
        out.append(d)
    out.sort(key=lambda d: -d["share"])
    top = out[0]
    tr = traffic.get((workload, top["kernel"]))
    hbm = {"bound": "hbm", "kernel": top["kernel"], "achieved": top["achieved_gbs"], "peak": hbm_peak,
           "unit": "GB/s", "frac": top["frac_hbm"], "traffic": tr,
           "peak_kind": ("measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback")}
    if wl["precision"] == "df64":
        # FP64-class arithmetic on the FP32 pipe: the same algorithmic FP64 flops, compared
        # with what the FP64 pipe could do at most
        roofline = dict(hbm, fp64_equivalent={"achieved": top["fp64_tflops"], "unit": "TFLOP/s",
                                              "fp64_pipe_peak": round(FP64_PEAK_TFLOPS, 4),
                                              "ratio_to_fp64_peak": top["frac_fp64"]})
    elif wl["precision"] == "fp64":
        roofline = {"bound": "alu", "kernel": top["kernel"], "achieved": top["fp64_tflops"],
                    "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s", "frac": top["frac_fp64"],
                    "traffic": tr, "peak_kind": "FP64 pipe: 152 SMs x 2 FMA/clk x 2 flops x 2.07 GHz",
                    "hbm_view": hbm}
    else:
        roofline = hbm
    roofline["instrumented_ms_per_step"] = round(total / steps, 4)
    roofline["instrumented_wall_s"] = round(wall, 3)
    return roofline, out


def e2e_run(abi, c, steps):
    """Same metric through the C ABI with pinned HOST buffers: every step copies psi in from
    host memory, steps once, and copies psi out to host memory, with dgpe_step_host (the
    copies of successive steps overlapped with the steps; the state alternates between two
    device buffers, each with its captured step).
    Timed on the host clock from the first call to dgpe_sync, which waits for the last
    output copy.  `serial_ms_per_step` is the same loop with the synchronous dgpe_set_psi /
    dgpe_step / dgpe_get_psi calls, for comparison."""
    import torch
    n = 1
    for s in c.shape:
        n *= s
    host_in = torch.empty(c.shape, dtype=c.cdtype, pin_memory=True)
    host_out = torch.empty(c.shape, dtype=c.cdtype, pin_memory=True)
    abi.dgpe_get_psi(c.ctx, host_in.data_ptr(), abi.DGPE_HOST)
    # one untimed call: it allocates the second buffer and the copy streams and captures
    # the step on that buffer
    abi.dgpe_step_host(c.ctx, host_in.data_ptr(), host_out.data_ptr(), 1)
    abi.dgpe_sync(c.ctx)
    torch.cuda.synchronize(c.device)
    t0 = time.perf_counter()
    for _ in range(steps):
        abi.dgpe_step_host(c.ctx, host_in.data_ptr(), host_out.data_ptr(), 1)
    abi.dgpe_sync(c.ctx)
    wall = time.perf_counter() - t0
    torch.cuda.synchronize(c.device)
    t1 = time.perf_counter()
    for _ in range(steps):
        abi.dgpe_set_psi(c.ctx, host_in.data_ptr(), abi.DGPE_HOST)
        abi.dgpe_step(c.ctx, 1)
        abi.dgpe_get_psi(c.ctx, host_out.data_ptr(), abi.DGPE_HOST)
    abi.dgpe_sync(c.ctx)
    serial = time.perf_counter() - t1
    nbytes = host_in.numel() * host_in.element_size()
    return {"value": n * steps / wall, "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "ms_per_step": round(wall * 1e3 / steps, 4), "steps": steps,
            "wall_s": round(wall, 3), "api": "dgpe_step_host", "timer": "host clock, to dgpe_sync",
            "serial_ms_per_step": round(serial * 1e3 / steps, 4)}


def cpu_baseline(wl, budget_s=20.0):
    """The FP64 oracle, as it stands, on the host cores: whole SSCN steps of the same
    workload (grid, physics) until about `budget_s` seconds of CPU work."""
    import oracle
    from paper_1610_05329_gb300 import inputs
    p = oracle.make_params(wl["shape"], wl["h"], wl["dt"], oracle.REAL_TIME, wl["nu"], wl["g"], wl["gdd"])
    psi = inputs.gaussian_psi(wl["shape"], wl["h"], noise=1e-3, seed=1)
    n = psi.size
    steps, t = 0, 0.0
    while t < budget_s and steps < 1000:
        t0 = time.perf_counter()
        psi = oracle.step(p, psi, 1)
        t += time.perf_counter() - t0
        steps += 1
    return {"value": n * steps / t, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d full SSCN step(s) of the %dx%dx%d FP64 real-time workload, %.1f s" % (
                steps, *wl["shape"], t)}


def differentiation_run(abi, local, precision, steps, full=True):
    """The differentiation workload on 128^3 (h = 0.2, nu = (1, 1, nu_z(t)), g = 30,
    gdd = 15, real time dt = 0.001): forward step vs adjoint step time (CUDA events), and
    the whole sqrt(N)-checkpointed gradient of <z^2> over 50 segments x 40 steps with nu_z
    drawn from U[0.8, 1.2] (SplitMix64, seed 4)."""
    import torch
    from paper_1610_05329_gb300 import inputs
    shape, h = (128, 128, 128), 0.2
    prec = abi.DGPE_FP64 if precision == "fp64" else abi.DGPE_MIXED
    c = abi.Condensate(shape, h, 0.001, mode=abi.DGPE_IMAG_TIME, precision=prec, nu=(1.0, 1.0, 1.0), g=30.0,
                       gdd=15.0, device=torch.device("cuda", local))
    c.set_psi(torch.from_numpy(inputs.gaussian_psi(shape, h, noise=1e-3, seed=1)).to(device=c.device, dtype=c.cdtype))
    c.step(PREP_STEPS)
    c.set_params(mode=abi.DGPE_REAL_TIME)
    c.step(3)
    fwd = time_steps(c, steps, lambda: None)
    psi_k = c.get_psi(host=False)
    gbar = psi_k.clone()
    for _ in range(3):
        c.adjoint_step(psi_k, gbar)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(c.device)
    e0.record(c.stream)
    for _ in range(steps):
        c.adjoint_step(psi_k, gbar)
    e1.record(c.stream)
    torch.cuda.synchronize(c.device)
    adj = e0.elapsed_time(e1)
    out = {"grid": list(shape), "dtype": "f64" if precision == "fp64" else MIXED_DTYPE,
           "forward_ms_per_step": round(fwd / steps, 4), "adjoint_ms_per_step": round(adj / steps, 4),
           "adjoint_over_forward": round(adj / fwd, 3)}
    if full:
        nu_z = inputs.uniform(4, 50, 0.8, 1.2)
        t0 = time.perf_counter()
        loss, dnu, dg, dgdd = c.grad_z2(nu_z, 40)
        wall = time.perf_counter() - t0
        out.update({"grad_2000_steps_s": round(wall, 3), "grad_ms_per_step": round(wall / 2000 * 1e3, 4),
                    "grad_over_forward": round(wall / 2000 * 1e3 / (fwd / steps), 3), "loss_z2": loss,
                    "dL_dg": dg, "dL_dgdd": dgdd, "checkpoints": "sqrt(N): every 45 steps"})
    c.close()
    return out


def batching_run(abi, local, steps=300, count=64):
    """The batching workload: 64 independent imaginary-time FP32-mixed condensates, cube
    sizes drawn from {32, 48, 64, 96, 128} (SplitMix64 seed 5), h = 12.8/N, g ~ U[5, 80],
    gdd ~ U[0, 0.9 g], nu_d ~ U[0.5, 2], dt = 0.001, `steps` steps each.  Sequential
    per-condensate graph launches vs one batched graph launch for all `steps` steps (one
    chain of steps per member, joined once), after autotuning one member per distinct size;
    the first batched call (graph capture and instantiation, then the run) is untimed."""
    import torch
    from paper_1610_05329_gb300 import inputs
    sizes = [32, 48, 64, 96, 128]
    u = inputs.uniform(5, 6 * count)
    members = []
    for k in range(count):
        n = sizes[min(int(u[6 * k] * 5), 4)]
        g = 5.0 + 75.0 * u[6 * k + 1]
        gdd = 0.9 * g * u[6 * k + 2]
        nu = tuple(0.5 + 1.5 * u[6 * k + 3 + d] for d in range(3))
        members.append(dict(n=n, h=12.8 / n, g=g, gdd=gdd, nu=nu))
    conds, psis = [], []
    for k, m in enumerate(members):
        shape = (m["n"],) * 3
        c = abi.Condensate(shape, m["h"], 0.001, mode=abi.DGPE_IMAG_TIME, precision=abi.DGPE_MIXED, nu=m["nu"],
                           g=m["g"], gdd=m["gdd"], device=torch.device("cuda", local))
        psi = torch.from_numpy(inputs.gaussian_psi(shape, m["h"], noise=1e-3, seed=100 + k)).to(
            device=c.device, dtype=c.cdtype)
        conds.append(c)
        psis.append(psi)
        c.set_psi(psi)
    npts = sum(m["n"] ** 3 for m in members)
    tunings = {}
    for c, m in zip(conds, members):
        if m["n"] not in tunings:
            tunings[m["n"]] = c.autotune()
        else:
            c.set_tuning(tunings[m["n"]])
    st = torch.cuda.current_stream(conds[0].device)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    for c in conds:                      # warm-up (graph capture) of the sequential path
        c.step(1)
    for c, psi in zip(conds, psis):
        c.set_psi(psi)
    seq_ms = timed(lambda: [c.step(steps) for c in conds])
    b = abi.Batch(conds)
    t0 = time.perf_counter()
    b.step(steps)                        # builds the graph of `steps` steps per member, and runs it
    b.sync()
    first_call_s = time.perf_counter() - t0
    for c, psi in zip(conds, psis):
        c.set_psi(psi)
    torch.cuda.nvtx.range_push("batched")   # (profilers select the batched launch by this range)
    bat_ms = timed(lambda: b.step(steps))
    torch.cuda.nvtx.range_pop()
    b.sync()
    b.close()
    for c in conds:
        c.close()
    return {"condensates": count, "sizes": {str(n): sum(1 for m in members if m["n"] == n) for n in sizes},
            "steps": steps, "points": npts, "dtype": MIXED_DTYPE,
            "sequential_ms": round(seq_ms, 3), "batched_ms": round(bat_ms, 3),
            "sequential_updates_per_s": npts * steps / (seq_ms * 1e-3),
            "batched_updates_per_s": npts * steps / (bat_ms * 1e-3),
            "batched_speedup": round(seq_ms / bat_ms, 3),
            "batched_graph_launches": 1,
            "batched_first_call_s": round(first_call_s, 3),
            "autotune": {str(n): {k: (list(v) if isinstance(v, tuple) else v) for k, v in t.items()}
                         for n, t in tunings.items()}}


# The paper's own 3D timing grids and times for 1000 iterations (its Tables 1-3; precision
# unstated (C doubles), physics unstated): context only.
PAPER_GRIDS = {
    "480x480x480": {"shape": (480, 480, 480), "paper": "Table 1: imag3d-th 888 s, real3d-th 1466 s (16 cores, T=16)"},
    "480x480x500": {"shape": (480, 480, 500), "paper": "Table 2: imag3d-mpi 1124 s (1 node) / 96 s (32 nodes); real3d-mpi 2140 / 129 s"},
    "480x480x250": {"shape": (480, 480, 250), "paper": "Table 3: imag3d CUDA 579 s, real3d CUDA 800 s (1 Tesla M2090); 61 / 80 s on 32 GPUs"},
}


def paper_grid_run(abi, local, steps=5):
    """FP64 imaginary- and real-time steps on the paper's timing grids (h = 0.05, trap
    (1, 1, 1.5), g = 40, gdd = 20, dt = 5e-4): ms/step and the time of 1000 iterations."""
    import torch
    from paper_1610_05329_gb300 import inputs
    out = {}
    for name, spec in PAPER_GRIDS.items():
        shape = spec["shape"]
        c = abi.Condensate(shape, 0.05, 5e-4, mode=abi.DGPE_IMAG_TIME, nu=(1.0, 1.0, 1.5), g=40.0, gdd=20.0,
                           device=torch.device("cuda", local))
        c.set_psi(torch.from_numpy(inputs.gaussian_psi(shape, 0.05, noise=1e-3, seed=1)).to(device=c.device,
                                                                                            dtype=c.cdtype))
        c.step(2)
        ms_imag = time_steps(c, steps, lambda: None) / steps
        c.set_params(mode=abi.DGPE_REAL_TIME)
        c.step(2)
        ms_real = time_steps(c, steps, lambda: None) / steps
        c.close()
        npts = shape[0] * shape[1] * shape[2]
        out[name] = {"imag_ms_per_step": round(ms_imag, 3), "real_ms_per_step": round(ms_real, 3),
                     "imag_1000_steps_s": round(ms_imag, 3), "real_1000_steps_s": round(ms_real, 3),
                     "real_updates_per_s": npts / (ms_real * 1e-3), "paper": spec["paper"]}
    return out


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed on the host cores (rank 0 only)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1610_05329_gb300 import inputs
    wl = WORKLOADS["real256_fp64"]
    p = oracle.make_params(wl["shape"], wl["h"], wl["dt"], oracle.REAL_TIME, wl["nu"], wl["g"], wl["gdd"])
    psi = inputs.gaussian_psi(wl["shape"], wl["h"], noise=1e-3, seed=1)
    n = psi.size
    t0 = time.perf_counter()
    psi = oracle.step(p, psi, 1)        # the first untimed warm-up step sizes the run
    t_step = time.perf_counter() - t0
    cap = max(1, int(150.0 / max(t_step, 1e-3)))
    warmup = max(1, min(args.warmup, cap))
    if warmup > 1:
        psi = oracle.step(p, psi, warmup - 1)
    steps = min(args.steps, cap)
    t0 = time.perf_counter()
    psi = oracle.step(p, psi, steps)
    t = time.perf_counter() - t0
    value = n * steps / t
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": steps,
            "warmup": warmup, "ms_per_step": t / steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "real256_fp64", "grid": list(wl["shape"]), "mode": "real", "h": wl["h"],
                       "dt": wl["dt"], "g": wl["g"], "gdd": wl["gdd"], "nu": list(wl["nu"])},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "%d of %d requested full 256^3 FP64 steps after %d warm-up steps "
                                       "(each phase capped to ~150 s)" % (steps, args.steps, warmup)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle leg (profiling runs)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the 512x512x384 mixed-precision line item")
    ap.add_argument("--no-df64", action="store_true", help="skip the 256^3 double-float line item")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-adjoint", action="store_true", help="skip the 128^3 differentiation line item")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-condensate batching line item")
    ap.add_argument("--batch-steps", type=int, default=300, help="steps of the batching line item")
    ap.add_argument("--no-paper-grids", action="store_true", help="skip the paper-grid context line item")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the 512x512x384 mixed-vs-FP64 error table (500 + 500 steps, and the oracle)")
    ap.add_argument("--no-ground-state", action="store_true",
                    help="skip the converged 256^3 ground state, quench and 1000 real-time steps")
    ap.add_argument("--workload", default=None, choices=sorted(WORKLOADS),
                    help="time only this workload (profiling); the default line times both")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.warmup < 3:
        args.warmup = 3

    import torch
    from paper_1610_05329_gb300 import abi, build
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        barrier = lambda: dist.barrier(device_ids=[local])
    else:
        torch.cuda.set_device(local)
        dist = None
        barrier = lambda: None
    if rank == 0 or ws == 1:
        build.build()
    if dist is not None:
        barrier()
    abi.load()
    hbm_peak, peak_kind = measured_peaks()

    name = args.workload or "real256_fp64"
    wl = WORKLOADS[name]
    if args.workload is not None:
        args.no_mixed = True
        args.no_df64 = True
    c = make_condensate(abi, wl, local)
    npts = wl["shape"][0] * wl["shape"][1] * wl["shape"][2]
    c.step(args.warmup)
    obs0 = c.observables()   # outside the timed region (it synchronises)
    clocks = ClockSampler(local)
    clocks.start()
    ms = time_steps(c, args.steps, barrier)
    clk = clocks.stop()
    physics = track_physics(obs0, c.observables(), args.steps)
    value, ms = aggregate_over_ranks(ms, npts * args.steps, dist, c.device)
    launches_per_step = c.step_launches()
    roofline, kernels = kernel_profile(c, min(args.steps, 50), hbm_peak, peak_kind, name)
    e2e = e2e_run(abi, c, args.e2e_steps) if args.e2e_steps > 0 else None
    c.sync()
    c.close()

    mixed = None
    if not args.no_mixed:
        wlm = WORKLOADS["real512x512x384_mixed"]
        cm = make_condensate(abi, wlm, local)
        nm = wlm["shape"][0] * wlm["shape"][1] * wlm["shape"][2]
        cm.step(args.warmup)
        msm = time_steps(cm, args.steps, barrier)
        value_m, msm = aggregate_over_ranks(msm, nm * args.steps, dist, cm.device)
        rl_m, kernels_m = kernel_profile(cm, min(args.steps, 50), hbm_peak, peak_kind, "real512x512x384_mixed")
        cm.sync()
        cm.close()
        mixed = {"value": value_m, "unit": UNIT, "ms_per_step": round(msm / args.steps, 4),
                 "dtype": MIXED_DTYPE, "grid": list(wlm["shape"]), "roofline": rl_m, "kernels": kernels_m,
                 "algorithmic_bytes_per_step": sum(k["bytes_per_launch"] * k["launches"] for k in kernels_m)
                 / min(args.steps, 50)}

    dfl = None
    if not args.no_df64:
        wld = WORKLOADS["real256_df64"]
        cd = make_condensate(abi, wld, local)
        nd = wld["shape"][0] * wld["shape"][1] * wld["shape"][2]
        cd.step(args.warmup)
        msd = time_steps(cd, args.steps, barrier)
        value_d, msd = aggregate_over_ranks(msd, nd * args.steps, dist, cd.device)
        rl_d, kernels_d = kernel_profile(cd, min(args.steps, 50), hbm_peak, peak_kind, "real256_df64")
        cd.sync()
        cd.close()
        dfl = {"value": value_d, "unit": UNIT, "ms_per_step": round(msd / args.steps, 4),
               "dtype": "df64 (pairs of FP32, ~48 significant bits; parity with the FP64 oracle <= 1e-10)",
               "grid": list(wld["shape"]), "roofline": rl_d, "kernels": kernels_d}

    diff = None
    if not args.no_adjoint and args.workload is None:
        diff = {p: differentiation_run(abi, local, p, min(args.steps, 50)) for p in ("fp64", "mixed")}

    batch = None
    if not args.no_batch and args.workload is None:
        batch = batching_run(abi, local, steps=args.batch_steps)
    paper = None
    if not args.no_paper_grids and args.workload is None:
        paper = paper_grid_run(abi, local)
    prec_table = None
    if not args.no_precision and args.workload is None and rank == 0:
        prec_table = precision_table(abi, local)
    ground = None
    if not args.no_ground_state and args.workload is None and rank == 0:
        ground = ground_state_run(abi, local)

    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Gaussian + SplitMix64 noise)",
            "config": {"workload": name, "grid": list(wl["shape"]), "mode": "real", "h": wl["h"],
                       "dt": wl["dt"], "g": wl["g"], "gdd": wl["gdd"], "nu": list(wl["nu"]),
                       "prep": "%d imaginary-time steps at g=%g from the seeded Gaussian" % (PREP_STEPS, wl["g_prep"]),
                       "l2": "inputs larger than L2 (psi %d MB > 129 MB)" % (npts * (8 if wl["precision"] == "mixed" else 16) >> 20),
                       "parallelism": "replicas" if ws > 1 else "1 GPU"},
            "gpu_launches": launches_per_step * args.steps, "clocks": clk, "roofline": roofline, "kernels": kernels, "e2e": e2e,
            "physics": physics}
    if mixed is not None:
        line["mixed_512x512x384"] = mixed
    if dfl is not None:
        line["df64_256"] = dfl
    if diff is not None:
        line["differentiation_128"] = diff
    if batch is not None:
        line["batching_64"] = batch
    if paper is not None:
        line["paper_grids_fp64"] = paper
    if prec_table is not None:
        line["precision_512x512x384"] = prec_table
    if ground is not None:
        line["ground_state_256"] = ground
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
