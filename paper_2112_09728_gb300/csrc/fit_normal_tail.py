"""Fits the coefficients of the kernels' upper normal tail (pg_device.cuh,
normal_tail): erfc(x) ~ t exp(-x^2 + Q(t - 0.66)), t = 1 / (1 + x/2), with Q
a degree-9 polynomial, fitted by iteratively reweighted least squares (a
step toward minimax) to log(erfc(x) / t) + x^2 on x in [0, 4.05] (the tail is
dropped past h = 5.66, x = h / sqrt 2 = 4.0). Prints the coefficients, the
fit's relative error and the absolute error of its binary32 evaluation on the
tail 0.5 erfc(x). Run by hand; the kernels hold its output as constants."""
import numpy as np
from scipy.special import erfc

T0, DEG = 0.66, 9


def fit():
    x = np.linspace(0.0, 4.05, 40001)
    t = 1.0 / (1.0 + 0.5 * x)
    target = np.log(erfc(x) / t) + x * x
    A = np.vander(t - T0, DEG + 1, increasing=True)
    w = np.ones_like(x)
    for _ in range(40):
        c, *_ = np.linalg.lstsq(A * w[:, None], target * w, rcond=None)
        err = A @ c - target
        w *= 1.0 + 50.0 * np.abs(err) / np.abs(err).max()
    return x, c, np.abs(err).max()


def binary32_tail(x, c):
    xf = x.astype(np.float32)
    t = (np.float32(1) / (np.float32(1) + np.float32(0.5) * xf)).astype(np.float32)
    s = (t - np.float32(T0)).astype(np.float32)
    q = np.zeros_like(s)
    for k in range(DEG, -1, -1):
        q = (q * s + np.float32(c[k])).astype(np.float32)
    e = (q - xf * xf).astype(np.float32)
    return 0.5 * t * np.exp2(e * np.float32(1.4426950408889634)).astype(np.float32)


if __name__ == "__main__":
    x, c, rel = fit()
    print("coefficients, constant term first:")
    print(", ".join("%.9ef" % v for v in c))
    tail = 0.5 * erfc(x.astype(np.float32).astype(np.float64))
    print("fit max relative error %.2e; binary32 tail max absolute error %.2e"
          % (rel, np.abs(binary32_tail(x, c) - tail).max()))
