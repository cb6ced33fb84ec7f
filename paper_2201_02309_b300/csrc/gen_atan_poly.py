"""Fit the odd polynomial used for arctan(t), |t| <= 1, in the backprojection.

atan(t) ~= t * P(t^2), P of degree n, fitted by iteratively reweighted least
squares towards the minimax (equioscillating) absolute error on [0, 1]
(Lawson's algorithm), in float64.  Prints the coefficients (highest degree
first, for Horner's scheme) and the max error of the float32 Horner
evaluation against numpy's float64 arctan.  The kernel's constants are this
script's output for n = 9.
"""
import sys

import numpy as np


def fit(n, iters=200):
    x = np.cos(np.linspace(0, np.pi / 2, 20001)) ** 1  # dense, clustered at both ends
    x = np.unique(np.concatenate([x, np.linspace(0, 1, 20001)]))
    s = x * x
    A = x[:, None] * s[:, None] ** np.arange(n + 1)[None, :]
    y = np.arctan(x)
    w = np.ones_like(x)
    for _ in range(iters):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(A * sw[:, None], y * sw, rcond=None)
        e = np.abs(A @ c - y)
        w = w * (e + 1e-300)
        w /= w.sum()
    return c, np.abs(A @ c - y).max()


def horner32(c, t):
    t = np.float32(t)
    s = t * t
    p = np.float32(c[-1])
    for k in range(len(c) - 2, -1, -1):
        p = np.float32(p * s + np.float32(c[k]))
    return t * p


if __name__ == "__main__":
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 9
    c, e64 = fit(n)
    t = np.linspace(-1, 1, 2000001).astype(np.float32)
    got = horner32(c, t).astype(np.float64)
    err = np.abs(got - np.arctan(t.astype(np.float64))).max()
    print(f"degree {2 * n + 1}: fit max abs error {e64:.3e}, float32 Horner max abs error {err:.3e}")
    for k in range(n, -1, -1):
        print(f"    {np.float32(c[k]).item():.9e}f,  // t^{2 * k + 1}")
