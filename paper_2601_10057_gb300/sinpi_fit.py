"""Coefficients of the FP32 sin(pi r), cos(pi r) polynomials of the stencil
kernel (``sincospi_<float>`` in ``csrc/step_kernels.cuh``).

For |r| <= 1/2: sin(pi r) = r P(r^2) with P of degree 4 (degree 9 in r) and
cos(pi r) = Q(r^2) with Q of degree 5 (degree 10 in r), fitted in FP64 by
least squares at Chebyshev nodes of [0, 1/2] and rounded to float.  Run
``python -m paper_2601_10057_gb300.sinpi_fit`` to print them.
"""
import numpy as np


def fit(nodes: int = 4000):
    t = np.cos(np.pi * (np.arange(nodes) + 0.5) / nodes) * 0.5
    r = t[t > 0]
    s = r * r

    def lsq(y, deg):
        A = np.vander(s, deg + 1, increasing=True)
        return np.linalg.lstsq(A, y, rcond=None)[0]

    return lsq(np.sin(np.pi * r) / r, 4), lsq(np.cos(np.pi * r), 5)


if __name__ == "__main__":
    cs, cc = fit()
    print("sin:", ", ".join(f"{np.float32(c):.9g}f" for c in cs))
    print("cos:", ", ".join(f"{np.float32(c):.9g}f" for c in cc))
