"""The kernels' rule for Z's corner integrals (the table in pg_params.cu,
fitted by fit_corner_rule.py). Each corner of Z adds the Drezner-Wesolowsky
correction I(h, k, rho) = 1/(2 pi) int_0^asin(rho) exp(-(h^2 + k^2 - 2 h k
sin t) / (2 cos^2 t)) dt to Phi(h) Phi(k), which the kernels take in s = sin t
on [0, rho] (dt = ds / sqrt(1 - s^2)) at nodes s = rho c with weights rho w;
the rule must integrate it, for every corner the kernels evaluate, about as
well as the 8-node Gauss-Legendre rule in t it replaced. Checked in binary64
against a 300-node Gauss-Legendre value in t on a seeded sample of live
corners (another sample than the fit's), and against Phi_2 itself through
Owen's T function at a few points, so that a wrong node, weight or sign in
the table fails."""
import os
import re

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2112_09728_gb300", "csrc")


def _table():
    src = open(os.path.join(CSRC, "pg_params.cu")).read()
    out = []
    for name in ("kZRuleC", "kZRuleW"):
        body = re.search(name + r"\[kZNodes\]\s*=\s*\{([^}]*)\}", src).group(1)
        out.append(np.array([float(v.strip().rstrip("f")) for v in body.split(",") if v.strip()]))
    n = int(re.search(r"constexpr int kZNodes = (\d+);", open(os.path.join(CSRC, "pg_device.cuh")).read()).group(1))
    assert len(out[0]) == len(out[1]) == n
    return out[0], out[1]


def _live_corners(seed, n):
    rng = np.random.default_rng(seed)
    h = rng.uniform(-6.5, 6.5, 4 * n)
    k = rng.uniform(-6.5, 6.5, 4 * n)
    r = rng.uniform(-0.9, 0.9, 4 * n)
    edge = rng.random(4 * n) < 0.25
    r[edge] = np.sign(r[edge]) * rng.uniform(0.8, 0.9, edge.sum())
    bound = np.where(h * k * r <= 0, h * h + k * k, np.maximum(h * h, k * k))
    keep = bound <= 36.0
    return h[keep][:n], k[keep][:n], r[keep][:n]


def _in_t(h, k, r, x, w):
    """A rule in t on [0, asin(rho)] given on [-1, 1] (nodes x, weights w)."""
    half = 0.5 * np.arcsin(r)
    t = half[:, None] * (1.0 + x[None, :])
    f = np.exp(-(h[:, None] ** 2 + k[:, None] ** 2 - 2.0 * h[:, None] * k[:, None] * np.sin(t))
               / (2.0 * np.cos(t) ** 2))
    return half * (f @ w) / (2.0 * np.pi)


def _rule(h, k, r, c, w):
    """The kernels' form: rho/(2 pi) sum w_i f(rho c_i) / sqrt(1 - (rho c_i)^2)."""
    s = r[:, None] * c[None, :]
    om = 1.0 - s * s
    f = np.exp(-(h[:, None] ** 2 + k[:, None] ** 2 - 2.0 * h[:, None] * k[:, None] * s) / (2.0 * om)) / np.sqrt(om)
    return r * (f @ w) / (2.0 * np.pi)


def test_rule_is_on_the_interval_and_integrates_the_arc():
    c, w = _table()
    assert np.all(np.diff(c) > 0) and c[0] > 0.0 and c[-1] < 1.0
    assert np.all(w > 0)
    # h = k = 0: the integrand in t is 1, the integral asin(rho) / (2 pi)
    r = np.linspace(-0.9, 0.9, 181)
    z = np.zeros_like(r)
    assert np.abs(_rule(z, z, r, c, w) - np.arcsin(r) / (2.0 * np.pi)).max() < 1.4e-8


def test_rule_matches_the_corner_integrals_within_the_replaced_rules_error():
    c, w = _table()
    h, k, r = _live_corners(2024, 40000)
    xr, wr = np.polynomial.legendre.leggauss(300)
    ref = _in_t(h, k, r, xr, wr)
    err = np.abs(_rule(h, k, r, c, w) - ref)
    x8, w8 = np.polynomial.legendre.leggauss(8)
    x6, w6 = np.polynomial.legendre.leggauss(len(c))
    err8 = np.abs(_in_t(h, k, r, x8, w8) - ref).max()
    err6 = np.abs(_in_t(h, k, r, x6, w6) - ref).max()
    assert err.max() < 1.6e-8, err.max()
    assert err.max() < 2.0 * err8 and err.max() < err6 / 20.0


def test_rule_gives_phi2_through_owens_t():
    """Phi_2(h, k; rho) = Phi(h) Phi(k) + I(h, k, rho) against the textbook
    Owen's T form (scipy's owens_t), at points spread over the live range."""
    sp = pytest.importorskip("scipy.special")
    c, w = _table()
    Phi = lambda v: 0.5 * sp.erfc(-v / np.sqrt(2.0))

    def phi2_owen(h, k, r):
        # Phi_2 = (Phi(h) + Phi(k))/2 - T(h, a_h) - T(k, a_k) - beta, with
        # a_h = (k - r h) / (h sqrt(1 - r^2)), a_k likewise, beta = 1/2 where
        # h k < 0 or (h k = 0 and h + k < 0), else 0
        s = np.sqrt(1.0 - r * r)
        ah, ak = (k - r * h) / (h * s), (h - r * k) / (k * s)
        beta = 0.5 if (h * k < 0 or (h * k == 0 and h + k < 0)) else 0.0
        return 0.5 * (Phi(h) + Phi(k)) - sp.owens_t(h, ah) - sp.owens_t(k, ak) - beta

    pts = [(0.3, 0.7, 0.5), (-1.2, 0.4, -0.8), (2.0, 1.5, 0.9), (-0.65, 0.76, 0.9), (0.7, -0.9, 0.9),
           (3.0, -2.5, -0.6), (-4.0, -3.5, 0.85), (1.1, 1.1, -0.9), (0.05, -0.2, 0.3), (5.5, 5.0, 0.9)]
    for h, k, r in pts:
        got = Phi(h) * Phi(k) + _rule(np.array([h]), np.array([k]), np.array([r]), c, w)[0]
        assert abs(got - phi2_owen(h, k, r)) < 2e-8, (h, k, r, got, phi2_owen(h, k, r))
