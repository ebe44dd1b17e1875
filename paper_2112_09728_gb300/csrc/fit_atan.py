"""Fits the coefficients of the kernels' arctangent on [-1, 1] (pg_device.cuh,
atan_unit, used by the inverse Shirley-Chiu map): (4/pi) atan(t) ~ t P(t^2)
with P of degree 7 (an odd polynomial of degree 15), fitted by iteratively
reweighted least squares (a step toward minimax) on t in [0, 1], the absolute
error being what the map needs (the square coordinate is r times it, r <= 1).
Prints the coefficients, the fit's absolute error and that of its binary32
evaluation by Horner's rule. Run by hand; the kernels hold its output as
constants."""
import numpy as np

DEG = 7


def fit():
    t = 0.5 + 0.5 * np.cos(np.linspace(0.0, np.pi, 20001))
    target = (4.0 / np.pi) * np.arctan(t)
    A = np.vander(t * t, DEG + 1, increasing=True) * t[:, None]
    w = np.ones_like(t)
    for _ in range(60):
        c, *_ = np.linalg.lstsq(A * w[:, None], target * w, rcond=None)
        err = A @ c - target
        w *= 1.0 + 50.0 * np.abs(err) / np.abs(err).max()
    tt = np.linspace(0.0, 1.0, 400001)
    e = (np.vander(tt * tt, DEG + 1, increasing=True) * tt[:, None]) @ c - (4.0 / np.pi) * np.arctan(tt)
    return c, np.abs(e).max()


def binary32(t, c):
    tf = t.astype(np.float32)
    t2 = (tf * tf).astype(np.float32)
    p = np.full_like(tf, np.float32(c[DEG]))
    for k in range(DEG - 1, -1, -1):
        p = (p * t2 + np.float32(c[k])).astype(np.float32)
    return (p * tf).astype(np.float32)


if __name__ == "__main__":
    c, err = fit()
    print("coefficients of t^1, t^3, ..., t^15:")
    print(", ".join("%.9ef" % v for v in c))
    t = np.linspace(-1.0, 1.0, 400001).astype(np.float32).astype(np.float64)
    ref = (4.0 / np.pi) * np.arctan(t)
    print("fit max absolute error %.2e; binary32 max absolute error %.2e" % (err, np.abs(binary32(t, c) - ref).max()))
