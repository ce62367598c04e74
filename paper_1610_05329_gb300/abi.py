"""Thin ctypes binding of the C ABI in include/dgpe.h (libdgpe.so).

Functions keep the C names and only marshal arguments; every step of the solver runs in
the CUDA kernels of the library.  ``Condensate`` is a convenience wrapper whose device
memory (the solver workspace) is a PyTorch tensor and whose stream is PyTorch's current
stream.  There is no fallback: if libdgpe.so is missing or fails to load, ``load()`` raises.
"""
import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdgpe.so")

DGPE_OK = 0
DGPE_EINVAL = -1
DGPE_ENOMEM = -2
DGPE_ECUDA = -3
DGPE_ENONFINITE = -4
DGPE_ETIMEOUT = -5
DGPE_EUNSUPPORTED = -6

DGPE_REAL_TIME = 0
DGPE_IMAG_TIME = 1
DGPE_FP64 = 0
DGPE_MIXED = 1
DGPE_DF64 = 2   # double-float pairs on the FP32 pipe; complex128 at the boundary
DGPE_HOST = 0
DGPE_DEVICE = 1
DGPE_SUB_POTENTIAL = 0
DGPE_SUB_CN_X = 1
DGPE_SUB_CN_Y = 2
DGPE_SUB_CN_Z = 3
DGPE_RECTANGLE = 0
DGPE_SIMPSON = 1
DGPE_KINETIC_LAPLACIAN3 = 0
DGPE_KINETIC_GRADIENT5 = 1


class dgpe_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("hx", ctypes.c_double), ("hy", ctypes.c_double), ("hz", ctypes.c_double),
                ("dt", ctypes.c_double), ("mode", ctypes.c_int), ("precision", ctypes.c_int),
                ("nu", ctypes.c_double * 3), ("g", ctypes.c_double), ("gdd", ctypes.c_double),
                ("cutoff", ctypes.c_double), ("integration", ctypes.c_int), ("kinetic", ctypes.c_int),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t)]


class dgpe_obs(ctypes.Structure):
    _fields_ = [("norm", ctypes.c_double), ("mu", ctypes.c_double), ("energy", ctypes.c_double),
                ("rms", ctypes.c_double * 3), ("e_kin", ctypes.c_double), ("e_trap", ctypes.c_double),
                ("e_contact", ctypes.c_double), ("e_dipolar", ctypes.c_double)]

    def as_dict(self):
        return {"norm": self.norm, "mu": self.mu, "energy": self.energy, "rms": tuple(self.rms),
                "e_kin": self.e_kin, "e_trap": self.e_trap, "e_contact": self.e_contact,
                "e_dipolar": self.e_dipolar}


class dgpe_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("total_ms", ctypes.c_double),
                ("launches", ctypes.c_longlong), ("bytes_per_launch", ctypes.c_double)]


class dgpe_tuning(ctypes.Structure):
    _fields_ = [("plan_style", ctypes.c_int * 3), ("ylines", ctypes.c_int), ("fft_threads", ctypes.c_int),
                ("cn_per_sm", ctypes.c_int), ("step_ms_default", ctypes.c_double), ("step_ms_tuned", ctypes.c_double)]

    def as_dict(self):
        return {"plan_style": tuple(self.plan_style), "ylines": self.ylines, "fft_threads": self.fft_threads,
                "cn_per_sm": self.cn_per_sm, "step_ms_default": self.step_ms_default,
                "step_ms_tuned": self.step_ms_tuned}

    @classmethod
    def from_dict(cls, d):
        t = cls()
        t.plan_style[0], t.plan_style[1], t.plan_style[2] = d["plan_style"]
        t.ylines, t.fft_threads, t.cn_per_sm = d["ylines"], d["fft_threads"], d["cn_per_sm"]
        return t


class DgpeError(RuntimeError):
    def __init__(self, code, what):
        msg = "%s: %s (%d)" % (what, strerror(code), code)
        if code == DGPE_ECUDA:
            msg += " [%s]" % dgpe_last_cuda_error()
        super().__init__(msg)
        self.code = code


_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every function declared in include/dgpe.h
_P = ctypes.POINTER
_SIGNATURES = [
    ("dgpe_workspace_bytes", ctypes.c_int, [_P(dgpe_params), _P(ctypes.c_size_t)]),
    ("dgpe_create", ctypes.c_int, [_P(dgpe_params), ctypes.c_void_p, _P(ctypes.c_void_p)]),
    ("dgpe_set_params", ctypes.c_int, [ctypes.c_void_p, _P(dgpe_params)]),
    ("dgpe_set_psi", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("dgpe_get_psi", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("dgpe_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("dgpe_step_host", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("dgpe_substep", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("dgpe_observables", ctypes.c_int, [ctypes.c_void_p, _P(dgpe_obs)]),
    ("dgpe_get_phi", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("dgpe_sync", ctypes.c_int, [ctypes.c_void_p]),
    ("dgpe_set_timing", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("dgpe_kernel_times", ctypes.c_int, [ctypes.c_void_p, _P(dgpe_kernel_time), ctypes.c_int, _P(ctypes.c_int)]),
    ("dgpe_adjoint_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("dgpe_adjoint_grads", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("dgpe_grad_z2_workspace_bytes", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _P(ctypes.c_size_t)]),
    ("dgpe_grad_z2", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_size_t, _P(ctypes.c_double), ctypes.c_void_p, _P(ctypes.c_double),
                                    _P(ctypes.c_double)]),
    ("dgpe_batch_create", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, _P(ctypes.c_void_p)]),
    ("dgpe_batch_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("dgpe_batch_sync", ctypes.c_int, [ctypes.c_void_p]),
    ("dgpe_batch_destroy", None, [ctypes.c_void_p]),
    ("dgpe_autotune", ctypes.c_int, [ctypes.c_void_p, _P(dgpe_tuning)]),
    ("dgpe_get_tuning", ctypes.c_int, [ctypes.c_void_p, _P(dgpe_tuning)]),
    ("dgpe_step_launches", ctypes.c_int, [ctypes.c_void_p, _P(ctypes.c_int)]),
    ("dgpe_set_tuning", ctypes.c_int, [ctypes.c_void_p, _P(dgpe_tuning)]),
    ("dgpe_moments_noalloc", ctypes.c_int, [ctypes.c_void_p, _P(dgpe_params), ctypes.c_void_p, ctypes.c_void_p]),
    ("dgpe_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("dgpe_last_cuda_error", ctypes.c_char_p, []),
    ("dgpe_destroy", None, [ctypes.c_void_p]),
]


def load():
    """Load libdgpe.so (built by paper_1610_05329_gb300.build); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libdgpe.so not found at %s: run paper_1610_05329_gb300/build.py "
                                   "(there is no CPU fallback)" % LIB_PATH)
            lib = ctypes.CDLL(LIB_PATH)
            for name, res, args in _SIGNATURES:
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
        return _lib


def _check(rc, what):
    if rc != DGPE_OK:
        raise DgpeError(rc, what)


def strerror(code):
    return load().dgpe_strerror(int(code)).decode()


def dgpe_last_cuda_error():
    return load().dgpe_last_cuda_error().decode()


def make_params(shape, h, dt, mode=DGPE_IMAG_TIME, precision=DGPE_FP64, nu=(1.0, 1.0, 1.0), g=0.0, gdd=0.0,
                workspace=None, workspace_bytes=0, cutoff=0.0, integration=DGPE_RECTANGLE,
                kinetic=DGPE_KINETIC_LAPLACIAN3):
    hx, hy, hz = (h, h, h) if np.isscalar(h) else tuple(h)
    p = dgpe_params()
    p.nx, p.ny, p.nz = (int(v) for v in shape)
    p.hx, p.hy, p.hz = float(hx), float(hy), float(hz)
    p.dt = float(dt)
    p.mode = int(mode)
    p.precision = int(precision)
    p.nu[0], p.nu[1], p.nu[2] = (float(v) for v in nu)
    p.g, p.gdd = float(g), float(gdd)
    p.cutoff = float(cutoff)
    p.integration = int(integration)
    p.kinetic = int(kinetic)
    p.workspace = workspace
    p.workspace_bytes = int(workspace_bytes)
    return p


# ---- raw C calls (return codes checked, names as in dgpe.h) ----------------------------
def dgpe_workspace_bytes(params):
    n = ctypes.c_size_t(0)
    _check(load().dgpe_workspace_bytes(ctypes.byref(params), ctypes.byref(n)), "dgpe_workspace_bytes")
    return n.value


def dgpe_create(params, stream=0):
    ctx = ctypes.c_void_p()
    _check(load().dgpe_create(ctypes.byref(params), ctypes.c_void_p(stream or None), ctypes.byref(ctx)),
           "dgpe_create")
    return ctx


def dgpe_set_params(ctx, params):
    _check(load().dgpe_set_params(ctx, ctypes.byref(params)), "dgpe_set_params")


def dgpe_set_psi(ctx, ptr, where):
    _check(load().dgpe_set_psi(ctx, ctypes.c_void_p(ptr), int(where)), "dgpe_set_psi")


def dgpe_get_psi(ctx, ptr, where):
    _check(load().dgpe_get_psi(ctx, ctypes.c_void_p(ptr), int(where)), "dgpe_get_psi")


def dgpe_step(ctx, nsteps):
    _check(load().dgpe_step(ctx, int(nsteps)), "dgpe_step")


def dgpe_step_host(ctx, in_ptr, out_ptr, nsteps):
    _check(load().dgpe_step_host(ctx, ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), int(nsteps)),
           "dgpe_step_host")


def dgpe_substep(ctx, which):
    _check(load().dgpe_substep(ctx, int(which)), "dgpe_substep")


def dgpe_observables(ctx):
    o = dgpe_obs()
    _check(load().dgpe_observables(ctx, ctypes.byref(o)), "dgpe_observables")
    return o.as_dict()


def dgpe_get_phi(ctx, ptr, where):
    _check(load().dgpe_get_phi(ctx, ctypes.c_void_p(ptr), int(where)), "dgpe_get_phi")


def dgpe_sync(ctx):
    _check(load().dgpe_sync(ctx), "dgpe_sync")


def dgpe_set_timing(ctx, enable):
    _check(load().dgpe_set_timing(ctx, 1 if enable else 0), "dgpe_set_timing")


def dgpe_kernel_times(ctx, max_kernels=16):
    arr = (dgpe_kernel_time * max_kernels)()
    n = ctypes.c_int(0)
    _check(load().dgpe_kernel_times(ctx, arr, max_kernels, ctypes.byref(n)), "dgpe_kernel_times")
    return [{"name": arr[i].name.decode(), "total_ms": arr[i].total_ms, "launches": arr[i].launches,
             "bytes_per_launch": arr[i].bytes_per_launch} for i in range(min(n.value, max_kernels))]


def dgpe_adjoint_step(ctx, psi_k_ptr, gbar_ptr):
    _check(load().dgpe_adjoint_step(ctx, ctypes.c_void_p(psi_k_ptr), ctypes.c_void_p(gbar_ptr)), "dgpe_adjoint_step")


def dgpe_adjoint_grads(ctx, reset=False):
    out = (ctypes.c_double * 3)()
    _check(load().dgpe_adjoint_grads(ctx, out, 1 if reset else 0), "dgpe_adjoint_grads")
    return np.array(out[:])


def dgpe_grad_z2_workspace_bytes(ctx, nseg, steps_per_seg):
    n = ctypes.c_size_t(0)
    _check(load().dgpe_grad_z2_workspace_bytes(ctx, int(nseg), int(steps_per_seg), ctypes.byref(n)),
           "dgpe_grad_z2_workspace_bytes")
    return n.value


def dgpe_grad_z2(ctx, nu_z, steps_per_seg, work_ptr, work_bytes):
    nu = np.ascontiguousarray(nu_z, dtype=np.float64)
    dnu = np.zeros(nu.size)
    loss, dg, dgdd = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().dgpe_grad_z2(ctx, nu.size, int(steps_per_seg), nu.ctypes.data, ctypes.c_void_p(work_ptr),
                               int(work_bytes), ctypes.byref(loss), dnu.ctypes.data, ctypes.byref(dg),
                               ctypes.byref(dgdd)), "dgpe_grad_z2")
    return loss.value, dnu, dg.value, dgdd.value


def dgpe_autotune(ctx):
    t = dgpe_tuning()
    _check(load().dgpe_autotune(ctx, ctypes.byref(t)), "dgpe_autotune")
    return t.as_dict()


def dgpe_step_launches(ctx):
    n = ctypes.c_int()
    _check(load().dgpe_step_launches(ctx, ctypes.byref(n)), "dgpe_step_launches")
    return n.value


def dgpe_get_tuning(ctx):
    t = dgpe_tuning()
    _check(load().dgpe_get_tuning(ctx, ctypes.byref(t)), "dgpe_get_tuning")
    return t.as_dict()


def dgpe_set_tuning(ctx, tuning):
    t = dgpe_tuning.from_dict(tuning)
    _check(load().dgpe_set_tuning(ctx, ctypes.byref(t)), "dgpe_set_tuning")


def dgpe_batch_create(ctxs, stream=0):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    b = ctypes.c_void_p()
    _check(load().dgpe_batch_create(arr, len(ctxs), ctypes.c_void_p(stream or None), ctypes.byref(b)),
           "dgpe_batch_create")
    return b


def dgpe_batch_step(b, nsteps):
    _check(load().dgpe_batch_step(b, int(nsteps)), "dgpe_batch_step")


def dgpe_batch_sync(b):
    _check(load().dgpe_batch_sync(b), "dgpe_batch_sync")


def dgpe_batch_destroy(b):
    if b:
        load().dgpe_batch_destroy(b)


def dgpe_moments_noalloc(psi_ptr, params, out_ptr, stream=0):
    """Norm and rms sizes of a device psi into 4 device doubles, allocating nothing (for
    callers whose device memory is owned elsewhere or who must not allocate mid-run)."""
    _check(load().dgpe_moments_noalloc(ctypes.c_void_p(psi_ptr), ctypes.byref(params), ctypes.c_void_p(out_ptr),
                                       ctypes.c_void_p(stream or None)), "dgpe_moments_noalloc")


def dgpe_destroy(ctx):
    if ctx:
        load().dgpe_destroy(ctx)


# ---- convenience wrapper: PyTorch owns the device memory and the stream ----------------
class Condensate:
    """One solver context on the current CUDA device and PyTorch's current stream.

    psi arrays are [nx][ny][nz] complex128 (FP64, DF64) or complex64 (MIXED); numpy arrays are
    host memory, torch CUDA tensors device memory.
    """

    def __init__(self, shape, h, dt, mode=DGPE_IMAG_TIME, precision=DGPE_FP64, nu=(1.0, 1.0, 1.0),
                 g=0.0, gdd=0.0, device=None, cutoff=0.0, integration=DGPE_RECTANGLE,
                 kinetic=DGPE_KINETIC_LAPLACIAN3):
        import torch
        self._torch = torch
        self.shape = tuple(int(v) for v in shape)
        self.precision = precision
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        wide = precision != DGPE_MIXED   # FP64 and double-float exchange complex128
        self.cdtype = torch.complex128 if wide else torch.complex64
        self.rdtype = torch.float64 if wide else torch.float32
        self.np_cdtype = np.complex128 if wide else np.complex64
        self._params = make_params(shape, h, dt, mode, precision, nu, g, gdd, cutoff=cutoff,
                                   integration=integration, kinetic=kinetic)
        nbytes = dgpe_workspace_bytes(self._params)
        self._ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self._params.workspace = self._ws.data_ptr()
        self._params.workspace_bytes = nbytes
        self.stream = torch.cuda.current_stream(self.device)
        self.ctx = dgpe_create(self._params, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "ctx", None):
            dgpe_destroy(self.ctx)   # waits for the copies of dgpe_step_host
            self.ctx = None
            self._ws = None
            self._host_refs = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_params(self, **kw):
        p = self._params
        for k, v in kw.items():
            if k == "h":
                hx, hy, hz = (v, v, v) if np.isscalar(v) else tuple(v)
                p.hx, p.hy, p.hz = hx, hy, hz
            elif k == "nu":
                p.nu[0], p.nu[1], p.nu[2] = (float(x) for x in v)
            elif k in ("dt", "g", "gdd", "cutoff"):
                setattr(p, k, float(v))
            elif k in ("mode", "integration", "kinetic"):
                setattr(p, k, int(v))
            else:
                raise KeyError(k)
        dgpe_set_params(self.ctx, p)

    def set_psi(self, psi):
        torch = self._torch
        if isinstance(psi, torch.Tensor):
            t = psi.to(device=self.device, dtype=self.cdtype).contiguous()
            assert tuple(t.shape) == self.shape
            dgpe_set_psi(self.ctx, t.data_ptr(), DGPE_DEVICE)
            self._keep = t   # the copy is stream-ordered: keep the source alive
        else:
            a = np.ascontiguousarray(psi, dtype=self.np_cdtype)
            assert a.shape == self.shape
            dgpe_set_psi(self.ctx, a.ctypes.data, DGPE_HOST)

    def get_psi(self, host=True):
        if host:
            out = np.empty(self.shape, dtype=self.np_cdtype)
            dgpe_get_psi(self.ctx, out.ctypes.data, DGPE_HOST)
            return out
        out = self._torch.empty(self.shape, dtype=self.cdtype, device=self.device)
        dgpe_get_psi(self.ctx, out.data_ptr(), DGPE_DEVICE)
        return out

    def phi(self, host=True):
        if host:
            out = np.empty(self.shape, dtype=np.float32 if self.precision == DGPE_MIXED else np.float64)
            dgpe_get_phi(self.ctx, out.ctypes.data, DGPE_HOST)
            return out
        out = self._torch.empty(self.shape, dtype=self.rdtype, device=self.device)
        dgpe_get_phi(self.ctx, out.data_ptr(), DGPE_DEVICE)
        return out

    def step(self, nsteps=1):
        dgpe_step(self.ctx, nsteps)

    def step_host(self, psi_in, psi_out, nsteps=1):
        """dgpe_step_host on CPU tensors or arrays of psi's shape and boundary dtype
        (pinned tensors make the copies asynchronous).  Both must stay alive and unchanged,
        and psi_out unread, until sync()."""
        ptrs = []
        for t in (psi_in, psi_out):
            if isinstance(t, np.ndarray):
                assert t.shape == self.shape and t.dtype == self.np_cdtype and t.flags.c_contiguous
                ptrs.append(t.ctypes.data)
            else:
                assert tuple(t.shape) == self.shape and t.dtype == self.cdtype and t.is_contiguous()
                assert t.device.type == "cpu"
                ptrs.append(t.data_ptr())
        # the copies are asynchronous: hold the buffers of every call until sync()
        self._host_refs = getattr(self, "_host_refs", []) + [(psi_in, psi_out)]
        dgpe_step_host(self.ctx, ptrs[0], ptrs[1], nsteps)

    def substep(self, which):
        dgpe_substep(self.ctx, which)

    def observables(self):
        return dgpe_observables(self.ctx)

    def sync(self):
        dgpe_sync(self.ctx)
        self._host_refs = []

    def set_timing(self, enable):
        dgpe_set_timing(self.ctx, enable)

    def kernel_times(self):
        return dgpe_kernel_times(self.ctx)

    def autotune(self):
        return dgpe_autotune(self.ctx)

    def set_tuning(self, tuning):
        dgpe_set_tuning(self.ctx, tuning)

    def tuning(self):
        return dgpe_get_tuning(self.ctx)

    def step_launches(self):
        return dgpe_step_launches(self.ctx)

    def adjoint_step(self, psi_k, gbar):
        """gbar (device tensor) <- cotangent of psi_k for one real-time step (in place)."""
        dgpe_adjoint_step(self.ctx, psi_k.data_ptr(), gbar.data_ptr())

    def adjoint_grads(self, reset=False):
        return dgpe_adjoint_grads(self.ctx, reset)

    def grad_z2(self, nu_z, steps_per_seg):
        """(L, dL/dnu_z[nseg], dL/dg, dL/dgdd) of L = <z^2> of the final state of a real-time
        trajectory under a piecewise-constant nu_z schedule (sqrt(N) checkpointing); the
        checkpoint buffer is a PyTorch tensor kept between calls."""
        nu = np.ascontiguousarray(nu_z, dtype=np.float64)
        need = dgpe_grad_z2_workspace_bytes(self.ctx, nu.size, steps_per_seg)
        work = getattr(self, "_grad_work", None)
        if work is None or work.numel() < need:
            work = self._torch.empty(need, dtype=self._torch.uint8, device=self.device)
            self._grad_work = work
        return dgpe_grad_z2(self.ctx, nu, steps_per_seg, work.data_ptr(), work.numel())


class Batch:
    """Independent condensates advanced together by one CUDA graph per step (their kernels
    run as parallel graph branches) on PyTorch's current stream."""

    def __init__(self, condensates):
        import torch
        self.members = list(condensates)
        self.stream = torch.cuda.current_stream()
        self.handle = dgpe_batch_create([c.ctx for c in self.members], self.stream.cuda_stream)

    def step(self, nsteps=1):
        dgpe_batch_step(self.handle, nsteps)

    def sync(self):
        dgpe_batch_sync(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            dgpe_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trajectory_z2(condensate, nu_z, g, gdd, steps_per_seg):
    """Differentiable L = <z^2> of the final state of a real-time trajectory (torch autograd).

    nu_z: 1-D float64 tensor (one trap frequency per segment), g, gdd: 0-d float64 tensors.
    The trajectory starts from the condensate's current psi, which is restored afterwards.
    Gradients come from the hand-written adjoint (dgpe_grad_z2)."""
    return _TrajectoryZ2.apply(nu_z, g, gdd, condensate, steps_per_seg)


def _make_autograd_function():
    import torch

    class TrajectoryZ2(torch.autograd.Function):
        @staticmethod
        def forward(ctx, nu_z, g, gdd, condensate, steps_per_seg):
            condensate.set_params(g=float(g), gdd=float(gdd))
            loss, dnu, dg, dgdd = condensate.grad_z2(nu_z.detach().cpu().numpy(), steps_per_seg)
            ctx.save_for_backward(torch.as_tensor(dnu, dtype=torch.float64),
                                  torch.tensor(dg, dtype=torch.float64), torch.tensor(dgdd, dtype=torch.float64))
            return torch.tensor(loss, dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad_out):
            dnu, dg, dgdd = ctx.saved_tensors
            g = grad_out.to(torch.float64)
            return g * dnu, g * dg, g * dgdd, None, None

    return TrajectoryZ2


class _LazyFunction:
    _fn = None

    def apply(self, *args):
        if _LazyFunction._fn is None:
            _LazyFunction._fn = _make_autograd_function()
        return _LazyFunction._fn.apply(*args)


_TrajectoryZ2 = _LazyFunction()
