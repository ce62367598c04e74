"""Provenance of the constants of the kernels' own sine and cosine (the phase e^{-i theta} of
the potential step).  Every constant of sin_cos(double) and sin_cos(float) in the device
header is checked against its definition:
  * the short-angle fits (|x| <= 1/8 cubics, |x| <= 1/4 cosine quartic) equal what
    csrc/fit_sincos.py computes (least squares at Chebyshev nodes in u = x^2, 40 digits), and
    their approximation errors, with the coefficients as rounded doubles evaluated exactly,
    are within the bounds the comments state (mpmath's sin and cos as the truth);
  * the Taylor coefficients are (-1)^k / n! rounded to double (float for the FP32 routine);
  * the Cody-Waite pieces of pi/2 sum to pi/2 and the leading ones are short enough for
    k * piece to be exact; 2/pi is the rounded 2/pi.
"""
import importlib.util
import math
import os
import re

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1610_05329_gb300", "csrc")
NUM = r"(-?[0-9.]+(?:e[-+]?[0-9]+)?)f?"


def _source(signature, end_marker):
    text = open(os.path.join(CSRC, "dgpe_device.cuh")).read()
    start = text.index(signature)
    return text[start:text.index(end_marker, start + 1)]


def _chains(body, var):
    """Horner chains of `var` in order: lists of literals, highest coefficient first."""
    chains = []
    for m in re.finditer(r"\b(?:double|float) %s = %s;" % (var, NUM), body):
        chain = [float(m.group(1))]
        pos = m.end()
        step_re = re.compile(r"\s*%s = fmaf?\(%s, u, %s\);" % (var, var, NUM))
        while True:
            step = step_re.match(body, pos)
            if not step:
                break
            chain.append(float(step.group(1)))
            pos = step.end()
        chains.append(chain)
    return chains


@pytest.fixture(scope="module")
def fp64():
    body = _source("__device__ __forceinline__ void sin_cos(double x", "__device__ __forceinline__ void sin_cos(float x")
    return {"ps": _chains(body, "ps"), "pc": _chains(body, "pc"), "body": body}


@pytest.fixture(scope="module")
def fp32():
    body = _source("__device__ __forceinline__ void sin_cos(float x", "exp_r(double x)")
    return {"ps": _chains(body, "ps"), "pc": _chains(body, "pc"), "body": body}


@pytest.fixture(scope="module")
def fits():
    spec = importlib.util.spec_from_file_location("fit_sincos", os.path.join(CSRC, "fit_sincos.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.fits()


def taylor(k0, k1, odd, cast=float):
    """(-1)^k / (2k+1)! (odd) or (-1)^(k+1) / (2k+2)! (even) for k = k0..k1, highest first."""
    out = []
    for k in range(k0, k1 + 1):
        n = 2 * k + 1 if odd else 2 * k + 2
        sign = (-1) ** k if odd else (-1) ** (k + 1)
        out.append(cast(sign / math.factorial(n)))
    return out[::-1]


def test_fp64_fits_are_regenerated(fp64, fits):
    # branches in order: |x| <= 1/8, |x| <= 1/4, general
    assert fp64["ps"][0] == fits["sin_eighth"][::-1]
    assert fp64["pc"][0] == fits["cos_eighth"][::-1]
    assert fp64["pc"][1] == fits["cos_quarter"][::-1]


def test_fp64_taylor_coefficients(fp64):
    assert fp64["ps"][1] == taylor(1, 5, odd=True)          # sine through x^11 (|x| <= 1/4)
    assert fp64["ps"][2] == taylor(1, 8, odd=True)          # through r^17 (reduced argument)
    assert fp64["pc"][2] == taylor(0, 8, odd=False)         # cosine through r^18


def _max_error(coefs_high_first, kind, xmax, n=1500):
    worst_abs = worst_rel = mp.mpf(0)
    with mp.workdps(40):
        for i in range(1, n + 1):
            x = mp.mpf(xmax) * i / n
            u = x * x
            p = mp.mpf(0)
            for c in coefs_high_first:
                p = p * u + mp.mpf(c)
            if kind == "sin":
                got, want = x + x * u * p, mp.sin(x)
            else:
                got, want = 1 + u * p, mp.cos(x)
            e = abs(got - want)
            worst_abs = max(worst_abs, e)
            worst_rel = max(worst_rel, e / abs(want))
    return float(worst_abs), float(worst_rel)


def test_fp64_fit_error_bounds(fp64):
    # the stated bounds of the comments: below 2e-19 relative (sine) and 2e-18 absolute
    # (cosine) on |x| <= 1/8; below 5.2e-19 for the cosine quartic on |x| <= 1/4; the
    # Taylor sine through x^11 below 3e-18 absolute on |x| <= 1/4.  The general series drops
    # terms below 1e-19 on |r| <= pi/4 (r^19/19!, r^20/20!); with its coefficients rounded to
    # double (-1/6 is off by 9e-18) it stays below 5e-18, under a tenth of an ulp of sin(pi/4)
    assert _max_error(fp64["ps"][0], "sin", 0.125)[1] < 2e-19
    assert _max_error(fp64["pc"][0], "cos", 0.125)[0] < 2e-18
    assert _max_error(fp64["pc"][1], "cos", 0.25)[0] < 5.2e-19
    assert _max_error(fp64["ps"][1], "sin", 0.25)[0] < 3e-18
    assert _max_error(fp64["ps"][2], "sin", math.pi / 4)[0] < 5e-18
    assert _max_error(fp64["pc"][2], "cos", math.pi / 4)[0] < 5e-18


def test_fp64_evaluation_in_doubles(fp64):
    """The polynomials evaluated in FP64 (Horner, plain multiply-add here; the GPU fuses
    them) stay within a few units in the last place of the true values."""
    xs = np.linspace(-0.125, 0.125, 4001)
    u = xs * xs
    ps = np.zeros_like(xs)
    pc = np.zeros_like(xs)
    for c in fp64["ps"][0]:
        ps = ps * u + c
    for c in fp64["pc"][0]:
        pc = pc * u + c
    s = xs * u * ps + xs
    c = u * pc + 1.0
    with mp.workdps(30):
        ts = np.array([float(mp.sin(mp.mpf(v))) for v in xs])
        tc = np.array([float(mp.cos(mp.mpf(v))) for v in xs])
    assert np.max(np.abs(s - ts)) <= 2 * np.finfo(float).eps * 0.125
    assert np.max(np.abs(c - tc)) <= 2 * np.finfo(float).eps


def test_fp64_cody_waite_pieces(fp64):
    pieces = [float(v) for v in re.findall(r"r = fma\(-k, %s, (?:x|r)\);" % NUM, fp64["body"])]
    assert len(pieces) == 3
    with mp.workdps(50):
        total = sum(mp.mpf(v) for v in pieces)
        assert abs(total - mp.pi / 2) < mp.mpf(10) ** -36
    # the two leading pieces have at most 32 significant bits: k * piece is exact for |k| < 2^21
    for v in pieces[:2]:
        m, _ = math.frexp(v)
        assert (int(m * 2 ** 53) & ((1 << 21) - 1)) == 0
    two_over_pi = float(re.search(r"rint\(x \* %s\)" % NUM, fp64["body"]).group(1))
    with mp.workdps(40):
        assert two_over_pi == float(2 / mp.pi)


def test_fp32_constants(fp32):
    f32 = lambda v: float(np.float32(v))
    # FP32 routine: |x| <= 1/4 sine through x^7 and cosine through x^6, then (reduced
    # argument) sine through r^9 and cosine through r^10; every literal the float of 1/n!
    assert [f32(v) for v in fp32["ps"][0]] == taylor(1, 3, odd=True, cast=f32)
    assert [f32(v) for v in fp32["pc"][0]] == taylor(0, 2, odd=False, cast=f32)
    assert [f32(v) for v in fp32["ps"][1]] == taylor(1, 4, odd=True, cast=f32)
    assert [f32(v) for v in fp32["pc"][1]] == taylor(0, 4, odd=False, cast=f32)
    # the short branch's truncation: first omitted terms x^9/9! and x^8/8! at x = 1/4
    assert 0.25 ** 9 / math.factorial(9) < 1.1e-11 and 0.25 ** 8 / math.factorial(8) < 3.8e-10
    pieces = [f32(v) for v in re.findall(r"r = fmaf\(-k, %s, (?:x|r)\);" % NUM, fp32["body"])]
    assert len(pieces) == 3
    with mp.workdps(40):
        assert abs(sum(mp.mpf(v) for v in pieces) - mp.pi / 2) < mp.mpf(10) ** -21
        two_over_pi = f32(re.search(r"fmaf\(x, %s, 12582912.0f\)" % NUM, fp32["body"]).group(1))
        assert two_over_pi == f32(float(2 / mp.pi))
