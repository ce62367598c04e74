"""FP64 CPU oracle of the SSCN step of the 3D dipolar Gross-Pitaevskii equation.

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it; the CUDA library and its Python binding never import it, and the
two share no code.  The arithmetic lives in ``dgpe_oracle.c`` (plain C, FP64, recursive
Cooley-Tukey FFT, Thomas solver), which cites the readings it takes of the paper's
"Solution method" (split-step Crank-Nicolson, dipolar term by the convolution theorem).
This module only compiles it with gcc and marshals numpy arrays.

Every function here is pinned by ``tests/test_oracle_*.py`` against closed forms,
brute force and invariants; the interacting values of mu and E beyond the virial
identity are "parity unpinned" (the paper prints no physical result).
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dgpe_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

REAL_TIME = 0
IMAG_TIME = 1


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("hx", ctypes.c_double), ("hy", ctypes.c_double), ("hz", ctypes.c_double),
                ("dt", ctypes.c_double), ("mode", ctypes.c_int),
                ("nu", ctypes.c_double * 3), ("g", ctypes.c_double), ("gdd", ctypes.c_double),
                ("cutoff", ctypes.c_double), ("integration", ctypes.c_int), ("kinetic", ctypes.c_int)]


class Obs(ctypes.Structure):
    _fields_ = [("norm", ctypes.c_double), ("mu", ctypes.c_double), ("energy", ctypes.c_double),
                ("rms", ctypes.c_double * 3), ("e_kin", ctypes.c_double), ("e_trap", ctypes.c_double),
                ("e_contact", ctypes.c_double), ("e_dipolar", ctypes.c_double)]

    def as_dict(self):
        return {"norm": self.norm, "mu": self.mu, "energy": self.energy,
                "rms": tuple(self.rms), "e_kin": self.e_kin, "e_trap": self.e_trap,
                "e_contact": self.e_contact, "e_dipolar": self.e_dipolar}


def build(force=False):
    """Compile dgpe_oracle.c into oracle/_build/liboracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.POINTER
            dp = ctypes.c_void_p
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_cutoff_factor.restype = ctypes.c_double
            L.orc_cutoff_factor.argtypes = [ctypes.c_double]
            L.orc_norm.restype = ctypes.c_double
            L.orc_norm.argtypes = [ctypes.POINTER(Params), ctypes.c_void_p]
            for name, args in [("orc_fft", [dp, ctypes.c_int, ctypes.c_int]),
                               ("orc_dft", [dp, ctypes.c_int, ctypes.c_int]),
                               ("orc_fft3", [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
                               ("orc_dipolar_kernel", [P(Params), dp]),
                               ("orc_dipolar_phi", [P(Params), dp, dp]),
                               ("orc_dipolar_phi_direct", [P(Params), dp, dp]),
                               ("orc_thomas", [ctypes.c_int, dp, dp, dp, dp, dp]),
                               ("orc_potential_step", [P(Params), dp]),
                               ("orc_cn_sweep", [P(Params), dp, ctypes.c_int]),
                               ("orc_step", [P(Params), dp, ctypes.c_int]),
                               ("orc_observables", [P(Params), dp, P(Obs)]),
                               ("orc_adjoint_step", [P(Params), dp, dp, dp]),
                               ("orc_grad_z2", [P(Params), ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, dp])]:
                f = getattr(L, name)
                f.argtypes = args
                f.restype = None
            _lib = L
        return _lib


def num_threads():
    return lib().orc_num_threads()


def make_params(shape, h, dt, mode, nu, g, gdd, cutoff=0.0, integration=0, kinetic=0):
    """shape = (nx, ny, nz); h = scalar or (hx, hy, hz); mode = REAL_TIME / IMAG_TIME;
    cutoff = spherical cutoff radius of the dipolar interaction (<= 0: none)."""
    hx, hy, hz = (h, h, h) if np.isscalar(h) else tuple(h)
    p = Params()
    p.nx, p.ny, p.nz = (int(v) for v in shape)
    p.hx, p.hy, p.hz = float(hx), float(hy), float(hz)
    p.dt = float(dt)
    p.mode = int(mode)
    p.nu[0], p.nu[1], p.nu[2] = (float(v) for v in nu)
    p.g, p.gdd = float(g), float(gdd)
    p.cutoff = float(cutoff)
    p.integration = int(integration)
    p.kinetic = int(kinetic)
    return p


def _c128(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def fft(x, sign=-1):
    x = _c128(x).copy()
    lib().orc_fft(_ptr(x), x.size, sign)
    return x


def dft(x, sign=-1):
    x = _c128(x).copy()
    lib().orc_dft(_ptr(x), x.size, sign)
    return x


def fft3(x, sign=-1):
    x = _c128(x).copy()
    nx, ny, nz = x.shape
    lib().orc_fft3(_ptr(x), nx, ny, nz, sign)
    return x


def dipolar_kernel(p):
    ut = np.empty((p.nx, p.ny, p.nz), dtype=np.float64)
    lib().orc_dipolar_kernel(ctypes.byref(p), _ptr(ut))
    return ut


def dipolar_phi(p, n):
    n = np.ascontiguousarray(n, dtype=np.float64)
    phi = np.empty_like(n)
    lib().orc_dipolar_phi(ctypes.byref(p), _ptr(n), _ptr(phi))
    return phi


def dipolar_phi_direct(p, n):
    n = np.ascontiguousarray(n, dtype=np.float64)
    phi = np.empty_like(n)
    lib().orc_dipolar_phi_direct(ctypes.byref(p), _ptr(n), _ptr(phi))
    return phi


def thomas(lo, di, up, rhs):
    lo, di, up, rhs = (_c128(v) for v in (lo, di, up, rhs))
    x = np.empty_like(rhs)
    lib().orc_thomas(rhs.size, _ptr(lo), _ptr(di), _ptr(up), _ptr(rhs), _ptr(x))
    return x


def potential_step(p, psi):
    psi = _c128(psi).copy()
    lib().orc_potential_step(ctypes.byref(p), _ptr(psi))
    return psi


def cn_sweep(p, psi, axis):
    psi = _c128(psi).copy()
    lib().orc_cn_sweep(ctypes.byref(p), _ptr(psi), int(axis))
    return psi


def step(p, psi, nsteps=1):
    psi = _c128(psi).copy()
    lib().orc_step(ctypes.byref(p), _ptr(psi), int(nsteps))
    return psi


def observables(p, psi):
    psi = _c128(psi)
    o = Obs()
    lib().orc_observables(ctypes.byref(p), _ptr(psi), ctypes.byref(o))
    return o.as_dict()


def adjoint_step(p, psi_k, gbar):
    """Cotangent of the step input and (dL/dg, dL/dgdd, dL/dnu_z) of one real-time step."""
    psi_k = _c128(psi_k)
    g = _c128(gbar).copy()
    grads = np.zeros(3)
    lib().orc_adjoint_step(ctypes.byref(p), _ptr(psi_k), _ptr(g), _ptr(grads))
    return g, grads


def grad_z2(p, nu_z, steps_per_seg, psi0):
    """L = h^3 sum z^2 |psi_N|^2 under a piecewise-constant nu_z schedule and its adjoint
    gradient: returns (L, dL/dnu_z[nseg], dL/dg, dL/dgdd)."""
    nu_z = np.ascontiguousarray(nu_z, dtype=np.float64)
    psi0 = _c128(psi0)
    loss, dg, dgdd = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    dnu = np.zeros(nu_z.size)
    lib().orc_grad_z2(ctypes.byref(p), nu_z.size, int(steps_per_seg), _ptr(nu_z), _ptr(psi0),
                      ctypes.byref(loss), _ptr(dnu), ctypes.byref(dg), ctypes.byref(dgdd))
    return loss.value, dnu, dg.value, dgdd.value


def cutoff_factor(x):
    return lib().orc_cutoff_factor(float(x))


def norm(p, psi):
    psi = _c128(psi)
    return lib().orc_norm(ctypes.byref(p), _ptr(psi))
