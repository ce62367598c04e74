#!/usr/bin/env python3
"""Coefficients of the short-angle FP64 sine and cosine of the potential step.

The phase step's angles are small (|theta| <= 1/8 for almost every point of the usual
workloads), so the kernel evaluates sin and cos there by short polynomials in u = x^2:

    sin x = x + x u Ps(u),   Ps ~ (sin x / x - 1) / u,   cubic,   |x| <= 1/8
    cos x = 1 + u Pc(u),     Pc ~ (cos x - 1) / u,       cubic,   |x| <= 1/8
    cos x = 1 + u Qc(u),     Qc ~ (cos x - 1) / u,       quartic, |x| <= 1/4

Method: discrete least squares in u at 64 Chebyshev nodes of [0, X^2] (the nodes of the
Chebyshev-weighted continuous fit), solved by the normal equations in 40-digit arithmetic
(mpmath), each coefficient rounded to the nearest double.  Run this file to print the
constants as C; the kernel's copies must equal them (a CPU test checks that, and the error
bounds of the rounded polynomials against mpmath's sine and cosine).
"""
import mpmath as mp

NODES = 64
DIGITS = 40


def _lsq_chebyshev_nodes(f, umax, degree):
    with mp.workdps(DIGITS):
        us = [umax * (1 - mp.cos(mp.pi * (k + mp.mpf(1) / 2) / NODES)) / 2 for k in range(NODES)]
        a = mp.matrix(NODES, degree + 1)
        b = mp.matrix(NODES, 1)
        for i, u in enumerate(us):
            for j in range(degree + 1):
                a[i, j] = u ** j
            b[i] = f(u)
        c = mp.lu_solve(a.T * a, a.T * b)
        return [float(c[j]) for j in range(degree + 1)]


def _sin_kernel(u):
    r = mp.sqrt(u)
    return (mp.sin(r) / r - 1) / u


def _cos_kernel(u):
    return (mp.cos(mp.sqrt(u)) - 1) / u


def fits():
    """{name: coefficients c_0..c_d (Horner order is c_d first)}."""
    with mp.workdps(DIGITS):
        return {
            "sin_eighth": _lsq_chebyshev_nodes(_sin_kernel, mp.mpf(1) / 64, 3),
            "cos_eighth": _lsq_chebyshev_nodes(_cos_kernel, mp.mpf(1) / 64, 3),
            "cos_quarter": _lsq_chebyshev_nodes(_cos_kernel, mp.mpf(1) / 16, 4),
        }


if __name__ == "__main__":
    for name, c in fits().items():
        print("%s (Horner order):" % name)
        for v in reversed(c):
            print("  %r" % v)
