"""Coefficients of the FP32 arctangent used by the labeling kernel.

atan(x) / x is approximated on [0, 1] by 1 + c1 s + ... + cd s^d with s = x^2;
the constant term is held at 1 so that the relative error vanishes as x -> 0
(far triangles, whose tiny solid angles dominate the count, then carry no
systematic bias).  The coefficients minimise the maximum relative error by
Lawson's iteratively reweighted least squares (a discrete minimax method) on a
dense grid.  Run: python fit_atan.py [degree]  (the kernel uses degree 8).
"""
import sys

import numpy as np


def fit(deg: int, iters: int = 300):
    x = np.cos(np.linspace(0, np.pi / 2, 20000))
    x = np.sort(np.concatenate([x, np.linspace(0, 1, 20000)]))[1:]
    s = x * x
    f = np.arctan(x) / x
    A = np.stack([s ** k for k in range(1, deg + 1)], 1)
    b = f - 1.0
    w = np.ones_like(s)
    for _ in range(iters):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(A * sw[:, None], b * sw, rcond=None)
        r = np.abs(A @ c - b)
        w = w * (r + 1e-30)
        w /= w.sum()
    err = np.max(np.abs(A @ c - b) / f)
    return c, err


if __name__ == "__main__":
    d = int(sys.argv[1]) if len(sys.argv) > 1 else 7
    c, e = fit(d)
    print(f"degree {d}: max relative error {e:.3e}")
    for k, v in enumerate(c, 1):
        print(f"constexpr float kA{k} = {float(v)!r}f;")
