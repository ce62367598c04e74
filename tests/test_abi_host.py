"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
function include/dgpe.h declares, and rejects invalid parameters before any CUDA call."""
import ctypes
import os
import re

import pytest

from paper_1610_05329_gb300 import abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return abi.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "dgpe.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dgpe_\w+)\s*\(", text)))


def test_header_declares_the_api():
    names = declared_functions()
    for n in ["dgpe_create", "dgpe_set_params", "dgpe_set_psi", "dgpe_get_psi", "dgpe_step",
              "dgpe_observables", "dgpe_sync", "dgpe_strerror", "dgpe_destroy", "dgpe_workspace_bytes"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert {s[0] for s in abi._SIGNATURES} == set(declared_functions())


def test_strerror(lib):
    assert abi.strerror(0) == "ok"
    assert "invalid" in abi.strerror(abi.DGPE_EINVAL)
    assert abi.strerror(-999) == "unknown error code"


def params(**kw):
    base = dict(shape=(16, 16, 16), h=0.2, dt=0.004, mode=abi.DGPE_IMAG_TIME, precision=abi.DGPE_FP64,
                nu=(1, 1, 1), g=20, gdd=10)
    base.update(kw)
    return abi.make_params(**base)


def test_workspace_bytes(lib):
    n64 = abi.dgpe_workspace_bytes(params(shape=(64, 64, 64)))
    n32 = abi.dgpe_workspace_bytes(params(shape=(64, 64, 64), precision=abi.DGPE_MIXED))
    psi64 = 64 ** 3 * 16
    spec64 = 33 * 64 * 64 * 16
    ut64 = 33 * 64 * 64 * 8   # the FP64 dipolar kernel table on the half spectrum
    y64 = psi64               # the forward-elimination scratch of the per-line sweeps
    assert psi64 + spec64 + ut64 + y64 <= n64 < psi64 + spec64 + ut64 + y64 + (1 << 20)
    assert n32 < n64 * 0.4


@pytest.mark.parametrize("bad", [
    dict(shape=(5, 16, 16)), dict(shape=(16, 22, 16)), dict(shape=(16, 16, 2)), dict(shape=(1024, 16, 16)),
    dict(shape=(16, 16, 26)), dict(h=0.0), dict(h=(0.2, -0.1, 0.2)), dict(h=float("nan")), dict(dt=0.0),
    dict(dt=-0.01), dict(dt=float("inf")), dict(mode=2), dict(precision=7), dict(g=float("nan")),
    dict(nu=(1, float("inf"), 1)),
])
def test_create_rejects_invalid_parameters_without_touching_the_gpu(lib, bad):
    p = params(**bad)
    ctx = ctypes.c_void_p()
    rc = lib.dgpe_create(ctypes.byref(p), None, ctypes.byref(ctx))
    assert rc == abi.DGPE_EINVAL
    assert not ctx.value


def test_null_arguments(lib):
    assert lib.dgpe_create(None, None, None) == abi.DGPE_EINVAL
    assert lib.dgpe_step(None, 1) == abi.DGPE_EINVAL
    assert lib.dgpe_step_host(None, None, None, 1) == abi.DGPE_EINVAL
    assert lib.dgpe_sync(None) == abi.DGPE_EINVAL
    assert lib.dgpe_get_tuning(None, None) == abi.DGPE_EINVAL
    assert lib.dgpe_step_launches(None, None) == abi.DGPE_EINVAL
    lib.dgpe_destroy(None)
    n = ctypes.c_size_t()
    assert lib.dgpe_workspace_bytes(ctypes.byref(params(shape=(7, 8, 8))), ctypes.byref(n)) == abi.DGPE_EINVAL


def test_too_small_workspace_is_rejected(lib):
    p = params()
    p.workspace = 1 << 20
    p.workspace_bytes = 16
    ctx = ctypes.c_void_p()
    assert lib.dgpe_create(ctypes.byref(p), None, ctypes.byref(ctx)) == abi.DGPE_ENOMEM


def test_binding_constants_match_the_header():
    """Every #define value of include/dgpe.h is the binding's constant of the same name, and
    every error code has its own message."""
    text = open(os.path.join(ROOT, "include", "dgpe.h")).read()
    defines = dict(re.findall(r"#define (DGPE_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", text))
    assert len(defines) >= 20
    for name, value in defines.items():
        assert getattr(abi, name) == int(value), name
    codes = [int(v) for k, v in defines.items() if k == "DGPE_OK" or k.startswith("DGPE_E")]
    messages = [abi.strerror(code) for code in codes]
    assert len(set(messages)) == len(codes) and "unknown error code" not in messages


def test_every_declaration_cites_the_paper():
    """Each entry point's comment names the passage of the paper it implements (section
    names of the program summary: Nature of problem, Solution method, Summary of revisions,
    Additional comments) or says that the paper has no counterpart."""
    text = open(os.path.join(ROOT, "include", "dgpe.h")).read()
    body = text[text.index("typedef struct dgpe_params"):]
    missing = []
    prev = 0
    for m in re.finditer(r"^(?:int|void|const char \*)\s*(dgpe_\w+)\s*\(", body, flags=re.M):
        chunk = body[prev:m.start()]
        comments = " ".join(re.findall(r"/\*(.*?)\*/", chunk, flags=re.S))
        if "paper" not in comments.lower():
            missing.append(m.group(1))
        prev = body.index(";", m.end()) + 1
    assert not missing, missing
