"""The warp-path kernels store only (wn, a) per DCT pair and form b from a:
forward b = exp(-i pi/4) conj(a), inverse b = exp(+i pi/4) conj(a), for every
pair k >= 1 (where a carries the same normalisation factor as b).  Checked
here from the closed forms of the even/odd (Makhoul) DCT post- and
pre-processing twiddles, in FP64, and for the kernels' FP32 evaluation
((ax -+ ay) / sqrt 2 with a float 1/sqrt 2) within 2 ulp of the FP64 value."""
import numpy as np
import pytest


def _closed_forms(N):
    M = N // 2
    k = np.arange(1, M // 2 + 1, dtype=np.float64)
    th = np.pi * k / (2.0 * N)
    c1 = np.sqrt(2.0 / N)
    s1 = 1.0 / (M * c1)
    a_f = 0.5 * c1 * np.exp(-1j * th)
    b_f = 0.5 * c1 * np.exp(1j * (th - np.pi / 4))
    a_i = 0.5 * s1 * np.exp(1j * th)
    b_i = 0.5 * s1 * np.exp(1j * (np.pi / 4 - th))
    return a_f, b_f, a_i, b_i


@pytest.mark.parametrize("N", [128, 1024, 2048, 8192])
def test_b_is_rotated_conjugate_of_a(N):
    a_f, b_f, a_i, b_i = _closed_forms(N)
    assert np.allclose(np.exp(-1j * np.pi / 4) * np.conj(a_f), b_f, rtol=0, atol=1e-15 * np.abs(b_f).max())
    assert np.allclose(np.exp(1j * np.pi / 4) * np.conj(a_i), b_i, rtol=0, atol=1e-15 * np.abs(b_i).max())


@pytest.mark.parametrize("N", [128, 2048, 8192])
def test_float_formula_within_two_ulp(N):
    a_f, b_f, a_i, b_i = _closed_forms(N)
    h = np.float32(0.70710678118654752440)
    for a, b, inv in ((a_f, b_f, False), (a_i, b_i, True)):
        ax, ay = a.real.astype(np.float32), a.imag.astype(np.float32)
        if inv:
            bx, by = (ax + ay) * h, (ax - ay) * h
        else:
            bx, by = (ax - ay) * h, -(ax + ay) * h
        ulp = np.spacing(np.float32(np.abs(b).max()))
        assert np.abs(bx.astype(np.float64) - b.real).max() <= 2 * ulp
        assert np.abs(by.astype(np.float64) - b.imag).max() <= 2 * ulp
