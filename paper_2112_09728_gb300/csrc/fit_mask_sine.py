"""Fits the coefficients of the sine in the kernels' occlusion mask
(pg_device.cuh, versine_pi2): q(x) = sqrt(2) sin(pi x / 2) ~ x P(x^2) on
x in [0, 1/2] with P of degree 3 (an odd polynomial of degree 7), fitted by
iteratively reweighted least squares (a step toward minimax) on the relative
error, which stays bounded at x = 0 for an odd function. The kernels square
it: q(x)^2 = 2 sin^2(pi x / 2) = 1 - cos(pi x), the distance of |sin| or
|cos| from 1 with its relative precision kept near 0 (x is the distance of a
phase to the nearest extremum, reduced exactly on the device).
Prints the coefficients, the fit's error and that of its binary32 evaluation
by Horner's rule (of q and of q^2). Run by hand; the kernels hold its output
as constants."""
import numpy as np

DEG = 3


def target(x):
    return np.sqrt(2.0) * np.sin(0.5 * np.pi * x)


def fit():
    x = 0.25 + 0.25 * np.cos(np.linspace(0.0, np.pi, 20001))   # [0, 1/2], denser at the ends
    x = x[x > 1e-6]
    t = target(x)
    A = np.vander(x * x, DEG + 1, increasing=True) * x[:, None]
    w = 1.0 / t
    for _ in range(60):
        c, *_ = np.linalg.lstsq(A * w[:, None], t * w, rcond=None)
        err = (A @ c - t) / t
        w *= 1.0 + 50.0 * np.abs(err) / np.abs(err).max()
    xx = np.linspace(1e-6, 0.5, 400001)
    e = ((np.vander(xx * xx, DEG + 1, increasing=True) * xx[:, None]) @ c - target(xx)) / target(xx)
    return c, np.abs(e).max()


def binary32(x, c):
    xf = x.astype(np.float32)
    x2 = (xf * xf).astype(np.float32)
    p = np.full_like(xf, np.float32(c[DEG]))
    for k in range(DEG - 1, -1, -1):
        p = (p * x2 + np.float32(c[k])).astype(np.float32)
    return (p * xf).astype(np.float32)


if __name__ == "__main__":
    c, err = fit()
    print("coefficients of x^1, x^3, ..., x^%d:" % (2 * DEG + 1))
    print(", ".join("%.9ef" % v for v in c))
    c = np.array([float("%.9e" % v) for v in c])
    x = np.linspace(0.0, 0.5, 400001).astype(np.float32)
    x = x[x > 0].astype(np.float64)
    q = binary32(x, c)
    v = (q * q).astype(np.float32).astype(np.float64)
    rq = np.abs(q - target(x)) / target(x)
    vref = 2.0 * np.sin(0.5 * np.pi * x) ** 2
    rv = np.abs(v - vref) / vref
    print("fit max relative error %.2e; binary32 max relative error of q %.2e, of q^2 %.2e" % (err, rq.max(), rv.max()))
