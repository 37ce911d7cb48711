"""The FP32 sin/cos polynomials of csrc/trig_poly.cuh, refitted on the host.

The fit: Lawson's iteratively reweighted least squares, which converges to the
minimax (Chebyshev) approximation, on 400 Chebyshev nodes of [0, pi/4]:
    sin r = r + r^3 P(r^2),        P of degree 2, minimax relative error;
    cos r = 1 - r^2/2 + r^4 Q(r^2), Q of degree 2, minimax absolute error.
The test repeats it, rounds to FP32, and requires the constants in the source
to be those values (to 2 FP32 ulps), and checks the stated error bounds of the
source's constants in float64 arithmetic on a dense grid.
"""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1609_04493_gb300", "csrc", "trig_poly.cuh")


def _source_coefficients():
    text = open(SRC).read()
    ps = re.search(r"const float ps = fmaf\(fmaf\(([-+0-9.e]+)f, r2, ([-+0-9.e]+)f\), r2, "
                   r"([-+0-9.e]+)f\)", text)
    pc = re.search(r"const float pc = fmaf\(fmaf\(fmaf\(([-+0-9.e]+)f, r2, ([-+0-9.e]+)f\), r2, "
                   r"([-+0-9.e]+)f\),\s*r2, -0.5f\)", text)
    assert ps and pc, "polynomial lines not found"
    # highest degree first in the source; return lowest first
    sin_c = [float(ps.group(k)) for k in (3, 2, 1)]
    cos_c = [float(pc.group(k)) for k in (3, 2, 1)]
    return np.float32(sin_c), np.float32(cos_c)


def _lawson(A, f, w0, iters=300):
    w = np.full(len(f), 1.0 / len(f))
    for _ in range(iters):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(A * (sw * w0)[:, None], f * sw * w0, rcond=None)
        e = np.abs(A @ c - f) * w0
        w = w * e
        w /= w.sum()
    return c


def _refit():
    N, hi = 400, np.pi / 4
    x = (np.cos((2 * np.arange(N) + 1) * np.pi / (2 * N)) + 1) / 2 * hi
    cs = _lawson(np.stack([x ** 3, x ** 5, x ** 7], 1), np.sin(x) - x, 1 / np.sin(x))
    cc = _lawson(np.stack([x ** 4, x ** 6, x ** 8], 1), np.cos(x) - 1 + x * x / 2, np.ones(N))
    return np.float32(cs), np.float32(cc)


def _ulps(a, b):
    a = np.asarray(a, np.float32).view(np.int32).astype(np.int64)
    b = np.asarray(b, np.float32).view(np.int32).astype(np.int64)
    return np.abs(a - b)


def test_source_constants_are_the_refit():
    sin_src, cos_src = _source_coefficients()
    sin_fit, cos_fit = _refit()
    assert np.all(_ulps(sin_src, sin_fit) <= 2), (sin_src, sin_fit)
    assert np.all(_ulps(cos_src, cos_fit) <= 2), (cos_src, cos_fit)


def test_source_polynomials_meet_the_stated_bounds():
    p, q = (c.astype(np.float64) for c in _source_coefficients())
    r = np.linspace(1e-7, np.pi / 4, 400001)
    r2 = r * r
    s = r + r ** 3 * (p[0] + r2 * (p[1] + r2 * p[2]))
    c = 1 + r2 * (-0.5 + r2 * (q[0] + r2 * (q[1] + r2 * q[2])))
    assert np.max(np.abs(s / np.sin(r) - 1)) <= 9e-9
    assert np.max(np.abs(c - np.cos(r))) <= 6e-10
