"""The FP32 stencil's sin(pi x), cos(pi x) polynomials (the float
specialisation of sincospi_ in csrc/step_kernels.cuh): its constants are the
least-squares fit of sinpi_fit.py, and evaluated in float32 (no fused
multiply-add: a conservative stand-in for the device's FMA chain) they stay
within 2 ulp of 1 of sin and cos over |x| <= 4, exact at the integers."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2601_10057_gb300", "csrc", "step_kernels.cuh")


def _constants():
    src = open(HDR).read()
    body = src[src.index("void sincospi_<float>(float x"):]
    body = body[:body.index("\n}")]
    ps = [float(v) for v in re.findall(r"ps = fmaf\(q, (?:ps|[-0-9.e]+f), ([-0-9.e]+)f\)", body)]
    first_s = float(re.search(r"ps = fmaf\(q, ([-0-9.e]+)f,", body).group(1))
    pc = [float(v) for v in re.findall(r"pc = fmaf\(q, (?:pc|[-0-9.e]+f), ([-0-9.e]+)f\)", body)]
    first_c = float(re.search(r"pc = fmaf\(q, ([-0-9.e]+)f,", body).group(1))
    sin_c = list(reversed(ps)) + [first_s]     # ascending powers of q
    cos_c = list(reversed(pc)) + [first_c]
    return sin_c, cos_c


def _eval(x, sin_c, cos_c):
    x = np.asarray(x, np.float32)
    j = np.rint(x).astype(np.float32)
    r = (x - j).astype(np.float32)
    q = (r * r).astype(np.float32)
    ps = np.float32(sin_c[-1])
    for c in reversed(sin_c[:-1]):
        ps = (ps * q + np.float32(c)).astype(np.float32)
    pc = np.float32(cos_c[-1])
    for c in reversed(cos_c[:-1]):
        pc = (pc * q + np.float32(c)).astype(np.float32)
    sg = np.where((j.astype(np.int64) & 1) == 1, np.float32(-1), np.float32(1))
    return sg * (r * ps).astype(np.float32), sg * pc


def test_constants_are_the_fit():
    from paper_2601_10057_gb300.sinpi_fit import fit
    sin_c, cos_c = _constants()
    cs, cc = fit()
    assert len(sin_c) == 5 and len(cos_c) == 6
    assert np.array_equal(np.float32(sin_c), np.float32(cs))
    assert np.array_equal(np.float32(cos_c), np.float32(cc))


def test_error_within_two_ulp_of_one():
    sin_c, cos_c = _constants()
    x = np.linspace(-4.0, 4.0, 4_000_001).astype(np.float32)
    s, c = _eval(x, sin_c, cos_c)
    xd = x.astype(np.float64)
    ulp = float(np.spacing(np.float32(1.0)))
    assert np.abs(s - np.sin(np.pi * xd)).max() < 2 * ulp
    assert np.abs(c - np.cos(np.pi * xd)).max() < 2 * ulp


def test_exact_at_integers_and_half_integers():
    sin_c, cos_c = _constants()
    k = np.arange(-6, 7, dtype=np.float32)
    s, c = _eval(k, sin_c, cos_c)
    assert np.all(s == 0) and np.array_equal(c, np.where(k.astype(int) % 2 == 0, 1, -1).astype(np.float32))
    s2, _ = _eval(k + np.float32(0.5), sin_c, cos_c)
    assert np.allclose(np.abs(s2), 1.0, atol=2e-7, rtol=0)
