"""Writes oracle_imag64.txt: the FP64 oracle's state after the 64^3 imaginary-time workload
(h = 0.2, dt = 0.004, nu = (1, 1, 1), g = 20, gdd = 10, the seeded Gaussian with seed 1,
200 steps).  Calls only the oracle and the seeded input generator.  The values are a
regression fixture of the oracle itself; the GPU path is compared with them in
tests/test_golden.py."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

SHAPE, H, DT, NU, G, GDD, STEPS, SEED = (64, 64, 64), 0.2, 0.004, (1.0, 1.0, 1.0), 20.0, 10.0, 200, 1
KEYS = ("norm", "mu", "energy", "e_kin", "e_trap", "e_contact", "e_dipolar", "rms_x", "rms_y", "rms_z")


def compute():
    import oracle
    from paper_1610_05329_gb300 import inputs
    p = oracle.make_params(SHAPE, H, DT, oracle.IMAG_TIME, NU, G, GDD)
    psi = oracle.step(p, inputs.gaussian_psi(SHAPE, H, noise=1e-3, seed=SEED), STEPS)
    obs = dict(oracle.observables(p, psi))
    obs["rms_x"], obs["rms_y"], obs["rms_z"] = obs.pop("rms")
    return {k: obs[k] for k in KEYS}


if __name__ == "__main__":
    vals = compute()
    with open(os.path.join(HERE, "oracle_imag64.txt"), "w") as f:
        f.write("# written by tests/golden/make_oracle_golden.py (FP64 oracle, %d^3, %d imaginary-time steps)\n"
                % (SHAPE[0], STEPS))
        for k in KEYS:
            f.write("%-10s %.17g\n" % (k, vals[k]))
