"""Fits the quadrature rule of Z's corner integrals (pg_device.cuh, rect_mass).

Each corner of Z needs the Drezner-Wesolowsky correction of the bivariate
normal cdf,
    I(h, k, rho) = 1/(2 pi) int_0^asin(rho) exp(-(h^2 + k^2 - 2 h k sin t) / (2 cos^2 t)) dt
                 = 1/(2 pi) int_0^rho exp(-(h^2 + k^2 - 2 h k s) / (2 (1 - s^2))) / sqrt(1 - s^2) ds,
and the kernels take it in the second form by one fixed rule on [0, rho]:
s_i = rho c_i with weights rho w_i, so that a node needs neither the
arcsine of rho nor a sine, only 1/(1 - s^2) and its square root. Any fixed
(c_i, w_i) costs the same at run time, so instead of the Gauss-Legendre
nodes the rule is fitted to this family of integrands: the corners the
kernels evaluate, |rho| <= 0.9 (the guide's correlation clamp) and (h, k)
within the kernels' liveness bound (h^2 + k^2 <= 36 where h k rho <= 0,
max(h^2, k^2) <= 36 elsewhere). Six nodes fitted this way reach about the
worst-case absolute error of eight Gauss-Legendre nodes in t (six
Gauss-Legendre nodes in t are some 30 times worse, in s worse still).

Method: seeded samples of the family (30% of them with |rho| in [0.8, 0.9],
where the integrand is hardest), the exact integrals by a 300-node
Gauss-Legendre rule in t in binary64, the nodes through a logistic map so
that they stay inside (0, 1), the weights for given nodes by linear least
squares, the nodes by Levenberg-Marquardt on the residuals, and a reweighting
of the samples toward their largest errors after each fit (a step toward
minimax). The rule kept is the one with the smallest worst-case error on a
second, larger sample. Prints the rule in the kernels' form (c_i and w_i)
and the worst-case errors. Run by hand (a few minutes); pg_params.cu holds
its output as constants. The linear algebra runs on one thread, so that the
output does not depend on the order of a threaded library's reductions."""
import os

for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ[_v] = "1"

import numpy as np  # noqa: E402
from scipy.optimize import least_squares  # noqa: E402

N_NODES = 6
RHO_MAX = 0.9


def family(seed, n, edge_frac):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        h, k = rng.uniform(-6.5, 6.5, 2)
        r = rng.uniform(-RHO_MAX, RHO_MAX)
        if rng.random() < edge_frac:
            r = np.sign(r) * rng.uniform(0.8, RHO_MAX)
        bound = h * h + k * k if h * k * r <= 0 else max(h * h, k * k)
        if bound <= 36.0:
            out.append((h, k, r))
    return np.array(out)


def in_t(S, c):
    """Column i: T/(2 pi) times the integrand in t at t = T c_i, T = asin(rho)."""
    h, k, r = S.T
    T = np.arcsin(r)
    t = T[:, None] * c[None, :]
    f = np.exp(-(h[:, None] ** 2 + k[:, None] ** 2 - 2.0 * h[:, None] * k[:, None] * np.sin(t))
               / (2.0 * np.cos(t) ** 2))
    return (T / (2.0 * np.pi))[:, None] * f


def in_s(S, c):
    """Column i: rho/(2 pi) times the integrand in s at s = rho c_i."""
    h, k, r = S.T
    s = r[:, None] * c[None, :]
    om = 1.0 - s * s
    f = np.exp(-(h[:, None] ** 2 + k[:, None] ** 2 - 2.0 * h[:, None] * k[:, None] * s) / (2.0 * om)) / np.sqrt(om)
    return (r / (2.0 * np.pi))[:, None] * f


def exact(S):
    x, w = np.polynomial.legendre.leggauss(300)
    return in_t(S, (1.0 + x) / 2.0) @ (w / 2.0)


def gl_error(V, IV, n, form):
    x, w = np.polynomial.legendre.leggauss(n)
    return np.abs(form(V, (1.0 + x) / 2.0) @ (w / 2.0) - IV).max()


def fit(iters=25):
    S = family(11, 60000, 0.3)
    I = exact(S)
    V = family(12345, 200000, 0.2)
    IV = exact(V)
    x, _ = np.polynomial.legendre.leggauss(N_NODES)
    to_c = lambda z: 1.0 / (1.0 + np.exp(-z))
    z = np.log((1.0 + x) / (1.0 - x))            # the logistic map's inverse at (1 + x)/2
    wt = np.ones(len(I))
    best = (np.inf, None, None)
    for _ in range(iters):
        def res(zz):
            A = in_s(S, to_c(zz))
            w = np.linalg.lstsq(A * wt[:, None], I * wt, rcond=None)[0]
            return (A @ w - I) * wt
        z = least_squares(res, z, method="lm", xtol=1e-15, ftol=1e-15, max_nfev=3000).x
        c = to_c(z)
        A = in_s(S, c)
        w = np.linalg.lstsq(A * wt[:, None], I * wt, rcond=None)[0]
        e = np.abs(A @ w - I)
        ev = np.abs(in_s(V, c) @ w - IV).max()
        if ev < best[0]:
            best = (ev, c.copy(), w.copy())
        wt = wt * (e / e.max() + 0.02) ** 0.3
        wt /= wt.mean()
    ev, c, w = best
    o = np.argsort(c)
    return (c[o], w[o], ev, gl_error(V, IV, N_NODES, in_t), gl_error(V, IV, 8, in_t),
            gl_error(V, IV, N_NODES, in_s))


if __name__ == "__main__":
    c, w, ev, e6, e8, e6s = fit()
    print("worst-case absolute error on the validation sample: fitted %d nodes in s %.3e; Gauss-Legendre "
          "in t, %d nodes %.3e, 8 nodes %.3e; Gauss-Legendre in s, %d nodes %.3e"
          % (N_NODES, ev, N_NODES, e6, e8, N_NODES, e6s))
    print("c:", ", ".join("%.9ef" % v for v in c))
    print("w:", ", ".join("%.9ef" % v for v in w))
