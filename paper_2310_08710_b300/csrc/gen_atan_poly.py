"""Coefficients of atan2_poly (wsim_phases.cuh): atan(t) ~ t P(t^2) on [0, 1]
with P of degree 7, fitted for the smallest largest relative error by
Lawson's iteratively reweighted least squares (C. L. Lawson, 1961), then
rounded to float32.  Prints the coefficients (constant term first) and the
largest error of the float32 Horner evaluation on a dense grid.

    python paper_2310_08710_b300/csrc/gen_atan_poly.py
"""
import numpy as np


def fit(deg=7, iters=300):
    t = np.unique(np.concatenate([np.cos(np.linspace(0.0, np.pi / 2, 20001)), np.linspace(0.0, 1.0, 20001)]))[1:]
    s = t * t
    f = np.arctan(t) / t
    A = np.stack([s ** k for k in range(deg + 1)], 1)
    w = np.ones_like(t)
    for _ in range(iters):
        r = np.sqrt(w)
        c, *_ = np.linalg.lstsq(A * (r / f)[:, None], r, rcond=None)
        e = np.abs(A @ c / f - 1.0)
        w = w * e
        w /= w.sum()
    return c.astype(np.float32), float(e.max())


def horner32(c, t):
    s = (t * t).astype(np.float32)
    q = np.full_like(t, c[-1])
    for k in range(len(c) - 2, -1, -1):
        q = (q * s + c[k]).astype(np.float32)
    return (t * q).astype(np.float32)


if __name__ == "__main__":
    c, rel = fit()
    t = np.linspace(0.0, 1.0, 2000001).astype(np.float32)
    err = np.abs(horner32(c, t).astype(np.float64) - np.arctan(t.astype(np.float64))).max()
    print("coefficients:", ", ".join("%.9e" % v for v in c))
    print("largest relative error of the fit %.2e, absolute error of the float32 evaluation %.2e rad" % (rel, err))
