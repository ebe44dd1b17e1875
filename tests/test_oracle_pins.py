"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms, textbook special cases, brute force on
small inputs, or independent library routines (scipy). They are chosen so that
a dropped term, a wrong sign or index, or a transposed operand in the oracle
fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle as O
from paper_2112_09728_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Philox4x32-10 (random numbers of the guided draw, Sec. 3.1)
# ---------------------------------------------------------------------------
def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = O.philox(np.array([r[0:4]], np.uint32), np.array(r[4:6], np.uint32))
        assert [int(v) for v in out[0]] == r[6:10]


# ---------------------------------------------------------------------------
# Shirley-Chiu map M (Eq. 2)
# ---------------------------------------------------------------------------
def test_map_round_trip_and_unit_length():
    rng = np.random.default_rng(1)
    u = rng.uniform(0, 1, (2000, 2))
    w = O.square_to_hemi(u)
    assert np.allclose(np.linalg.norm(w, axis=1), 1.0, atol=1e-14)
    assert (w[:, 2] >= 0).all()
    assert np.abs(O.hemi_to_square(w) - u).max() < 1e-12


def test_map_boundary_centre_and_axes():
    assert np.allclose(O.square_to_hemi([0.5, 0.5])[0], [0, 0, 1])
    rng = np.random.default_rng(2)
    t = rng.uniform(0, 1, 50)
    edges = np.concatenate([np.stack([t, 0 * t], 1), np.stack([t, 0 * t + 1], 1),
                            np.stack([0 * t, t], 1), np.stack([0 * t + 1, t], 1)])
    assert np.abs(O.square_to_hemi(edges)[:, 2]).max() < 1e-14
    # the +x edge midpoint is the +x horizon direction, +y edge midpoint is +y
    assert np.allclose(O.square_to_hemi([1.0, 0.5])[0], [1, 0, 0], atol=1e-15)
    assert np.allclose(O.square_to_hemi([0.5, 1.0])[0], [0, 1, 0], atol=1e-15)


def test_map_constant_jacobian_2pi():
    rng = np.random.default_rng(3)
    h = 1e-6
    u = rng.uniform(0.01, 0.99, (3000, 2))
    a, b = 2 * u[:, 0] - 1, 2 * u[:, 1] - 1
    u = u[np.abs(np.abs(a) - np.abs(b)) > 1e-3]  # stay off the map's diagonal seams
    du = (O.square_to_hemi(u + [h, 0]) - O.square_to_hemi(u - [h, 0])) / (2 * h)
    dv = (O.square_to_hemi(u + [0, h]) - O.square_to_hemi(u - [0, h])) / (2 * h)
    jac = np.linalg.norm(np.cross(du, dv), axis=1)
    assert np.abs(jac / (2 * np.pi) - 1).max() < 1e-6


def test_map_uniform_square_gives_uniform_hemisphere_moments():
    n = 400
    g = (np.arange(n) + 0.5) / n
    U, V = np.meshgrid(g, g)
    w = O.square_to_hemi(np.stack([U.ravel(), V.ravel()], 1))
    # uniform on the hemisphere: E[z] = 1/2, E[z^2] = 1/3, E[x] = E[y] = 0, E[x^2] = 1/3
    assert abs(w[:, 2].mean() - 0.5) < 1e-5
    assert abs((w[:, 2] ** 2).mean() - 1 / 3) < 1e-5
    assert abs(w[:, 0].mean()) < 1e-12 and abs(w[:, 1].mean()) < 1e-12
    assert abs((w[:, 0] ** 2).mean() - 1 / 3) < 1e-5


def test_basis_orthonormal_right_handed():
    rng = np.random.default_rng(4)
    for _ in range(200):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        t, b = O.basis(n)
        m = np.stack([t, b, n])
        assert np.abs(m @ m.T - np.eye(3)).max() < 1e-12
        assert np.allclose(np.cross(t, b), n, atol=1e-12)
    t, b = O.basis([0, 0, 1])
    assert np.allclose(t, [1, 0, 0]) and np.allclose(b, [0, 1, 0])


# ---------------------------------------------------------------------------
# Normal distribution on the square and its mass Z
# ---------------------------------------------------------------------------
def _g5(mx, my, sx, sy, rho):
    return np.array([mx, my, sx * sx, sy * sy, rho * sx * sy])


def test_gauss_pdf_matches_scipy():
    rng = np.random.default_rng(5)
    for _ in range(50):
        g = _g5(*rng.uniform(0, 1, 2), *rng.uniform(0.01, 0.5, 2), rng.uniform(-0.9, 0.9))
        u = rng.uniform(-0.2, 1.2, 2)
        cov = [[g[2], g[4]], [g[4], g[3]]]
        ref = stats.multivariate_normal(g[:2], cov).pdf(u)
        assert O.gauss_pdf(g, u) == pytest.approx(ref, rel=1e-12, abs=1e-300)


def test_rect_mass_diagonal_is_product_of_1d_cdfs():
    rng = np.random.default_rng(6)
    gs = np.array([_g5(*rng.uniform(0, 1, 2), *np.exp(rng.uniform(-5, -0.5, 2)), 0.0)
                   for _ in range(40)])
    z = O.rect_mass(gs)
    sx, sy = np.sqrt(gs[:, 2]), np.sqrt(gs[:, 3])
    ref = (special.ndtr((1 - gs[:, 0]) / sx) - special.ndtr(-gs[:, 0] / sx)) * \
          (special.ndtr((1 - gs[:, 1]) / sy) - special.ndtr(-gs[:, 1] / sy))
    assert np.abs(z - ref).max() < 1e-12


def test_rect_mass_orthant_closed_form():
    # mean on the corner, spread tiny: Z -> P(X > 0, Y > 0) = 1/4 + asin(rho)/(2 pi)
    for rho in (-0.9, -0.5, 0.0, 0.3, 0.85):
        z = O.rect_mass(_g5(0.0, 0.0, 1e-3, 2e-3, rho))[0]
        assert z == pytest.approx(0.25 + math.asin(rho) / (2 * math.pi), abs=1e-11)
    # mean on an edge midpoint: half the mass
    assert O.rect_mass(_g5(0.0, 0.5, 1e-3, 1e-3, 0.7))[0] == pytest.approx(0.5, abs=1e-11)


def test_rect_mass_brute_force():
    """Midpoint sums on n x n and 2n x 2n grids, Richardson-extrapolated (the
    midpoint rule's error is c h^2 + O(h^4) for a smooth integrand)."""
    rng = np.random.default_rng(7)

    def brute(gg, n):
        g = (np.arange(n) + 0.5) / n
        U, V = np.meshgrid(g, g, indexing="ij")
        det = gg[2] * gg[3] - gg[4] ** 2
        dx, dy = U - gg[0], V - gg[1]
        q = (gg[3] * dx * dx - 2 * gg[4] * dx * dy + gg[2] * dy * dy) / det
        return np.exp(-0.5 * q).sum() / (n * n) / (2 * np.pi * np.sqrt(det))

    for _ in range(6):
        gg = _g5(*rng.uniform(0, 1, 2), *rng.uniform(0.08, 0.5, 2), rng.uniform(-0.9, 0.9))
        b1, b2 = brute(gg, 800), brute(gg, 1600)
        ref = (4 * b2 - b1) / 3
        assert O.rect_mass(gg)[0] == pytest.approx(ref, abs=2e-9)


def test_rect_mass_matches_scipy_bvn():
    rng = np.random.default_rng(8)
    for _ in range(10):
        gg = _g5(*rng.uniform(0, 1, 2), *rng.uniform(0.02, 0.6, 2), rng.uniform(-0.9, 0.9))
        cov = [[gg[2], gg[4]], [gg[4], gg[3]]]
        mvn = stats.multivariate_normal(gg[:2], cov, maxpts=10 ** 7, abseps=1e-12, releps=1e-12)
        ref = mvn.cdf([1, 1], lower_limit=[0, 0])
        assert O.rect_mass(gg)[0] == pytest.approx(ref, abs=1e-8)


def test_rect_mass_gradient_central_differences():
    rng = np.random.default_rng(9)
    gs = np.array([_g5(*rng.uniform(0.05, 0.95, 2), *rng.uniform(0.05, 0.5, 2),
                       rng.uniform(-0.8, 0.8)) for _ in range(12)])
    d = O.rect_mass_grad(gs)
    h = 1e-5
    for j in range(5):
        e = np.zeros(5)
        e[j] = h
        fd = (O.rect_mass(gs + e) - O.rect_mass(gs - e)) / (2 * h)
        assert np.abs(d[:, j] - fd).max() < 1e-6 * max(1.0, np.abs(fd).max())


# ---------------------------------------------------------------------------
# Materials
# ---------------------------------------------------------------------------
def _sph_quad(f, epsrel=1e-10):
    """Integral of f(w) over the upper hemisphere in (cos theta, phi)."""
    def g(c, phi):
        s = math.sqrt(max(0.0, 1 - c * c))
        return f(np.array([s * math.cos(phi), s * math.sin(phi), c]))
    v, _ = integrate.dblquad(g, 0, 2 * math.pi, 0, 1, epsabs=1e-11, epsrel=epsrel)
    return v


def test_lambert_pdf_normalised_and_sampler_consistent():
    wo = np.array([0.2, 0.1, math.sqrt(0.95)])
    assert _sph_quad(lambda w: O.brdf_pdf(-1.0, wo, w)) == pytest.approx(1.0, abs=1e-8)
    # f_r cos integrates to the albedo (energy conservation, exact for Lambert)
    assert _sph_quad(lambda w: O.brdf_cos(-1.0, 0.7, wo, w)) == pytest.approx(0.7, abs=1e-8)


def test_ggx_normal_distribution_normalised():
    # projected microfacet area: integral of D(h) cos(theta_h) over the hemisphere = 1;
    # probed through the pdf at normal incidence, where p_b = D(h) cos(h)/(4 cos(h))
    for rough in (0.3, 0.6, 1.0):
        wo = np.array([0.0, 0.0, 1.0])
        # at normal incidence the reflected direction is below the horizon only for
        # half vectors beyond 45 degrees; pdf over the upper hemisphere equals the
        # probability that the draw is valid
        tot = _sph_quad(lambda w: O.brdf_pdf(rough, wo, w), epsrel=1e-8)
        rng = np.random.default_rng(10)
        ok = np.mean([O.brdf_sample(rough, wo, *rng.uniform(0, 1, 2))[1] for _ in range(20000)])
        assert tot == pytest.approx(ok, abs=4 * math.sqrt(ok * (1 - ok) / 20000) + 1e-6)


def test_ggx_sampler_matches_pdf():
    rng = np.random.default_rng(11)
    for rough, wo in ((0.4, [0.3, -0.2, math.sqrt(0.87)]), (0.8, [0.6, 0.0, 0.8])):
        wo = np.array(wo)
        g = lambda w: w[0] ** 2 + 0.5 * w[2] + w[1] * w[2]
        ref = _sph_quad(lambda w: g(w) * O.brdf_pdf(rough, wo, w), epsrel=1e-8)
        n = 40000
        vals = np.zeros(n)
        for i in range(n):
            w, ok = O.brdf_sample(rough, wo, *rng.uniform(0, 1, 2))
            vals[i] = g(w) if ok else 0.0
        assert vals.mean() == pytest.approx(ref, abs=4 * vals.std() / math.sqrt(n))


def test_ggx_reciprocity_and_energy_bound():
    rng = np.random.default_rng(12)
    for _ in range(100):
        r = rng.uniform(0.02, 1.0)
        a = scenes.unit_hemisphere_dirs(rng, 2, zmin=0.05)
        f_ab = O.brdf_cos(r, 0.9, a[0], a[1]) / a[1][2]
        f_ba = O.brdf_cos(r, 0.9, a[1], a[0]) / a[0][2]
        assert f_ab == pytest.approx(f_ba, rel=1e-12)
    wo = np.array([0.5, 0.0, math.sqrt(0.75)])
    alb = _sph_quad(lambda w: O.brdf_cos(0.5, 1.0, wo, w), epsrel=1e-8)
    assert 0.5 < alb <= 1.0


# ---------------------------------------------------------------------------
# Radiance field
# ---------------------------------------------------------------------------
def test_vmf_lobe_normalised_on_sphere():
    for k in (5.0, 20.0, 80.0):
        f = O.make_field([[0.0, 0.0, 1.0]], [k], [1.0])
        # integrate over the full sphere in (cos theta, phi) around the lobe axis
        v, _ = integrate.quad(lambda c: O.radiance(f, [0, 0, 0], [math.sqrt(1 - c * c), 0, c]),
                              -1, 1, epsabs=1e-13, points=[1 - 1 / k])
        assert 2 * math.pi * v == pytest.approx(1.0, abs=1e-9)


# ---------------------------------------------------------------------------
# Mixture pdf, MIS, unbiasedness (Eq. 1, Eq. 2, Sec. 3.1)
# ---------------------------------------------------------------------------
def _one_pixel(rough=-1.0, normal=(0, 0, 1), albedo=0.8):
    g0 = np.array([[*normal, 2.0]], np.float32)
    g1 = np.array([[0, 0, rough, albedo]], np.float32)
    return g0, g1


def _gamma_row(mx, my, sxx, syy, sxy, pi, k=3.0, i=0.0):
    return np.array([[mx, my, sxx + mx * mx, syy + my * my, sxy + mx * my, pi, k, i]])


def _hemi_integral(cfg, cam, fld, g0, g1, gam, key, n):
    """2 pi * mean over an n x n midpoint grid of the square mapped by M (equal
    area), Richardson-extrapolated from n and 2n."""
    vals = []
    for m in (n, 2 * n):
        g = (np.arange(m) + 0.5) / m
        U, V = np.meshgrid(g, g)
        dirs = O.square_to_hemi(np.stack([U.ravel(), V.ravel()], 1))
        ev = O.evaluate(cfg, cam, fld, g0, g1, gam, dirs[:, None, :])
        vals.append(2 * np.pi * ev[key].mean())
    return (4 * vals[1] - vals[0]) / 3, ev


def test_mixture_pdf_integrates_to_one_lambert():
    cfg = O.make_config(1, 1)
    cam = O.make_camera(0, (0, 0, 5), (0, 0, -1), (1, 0, 0), (0, 1, 0))
    fld = O.make_field([[0, 0, 1]], [10.0], [1.0])
    g0, g1 = _one_pixel()
    for gam in (_gamma_row(0.3, 0.7, 0.01, 0.02, 0.005, 0.6),
                _gamma_row(0.02, 0.5, 0.05, 0.002, 0.0, 0.9),
                _gamma_row(0.5, 0.5, 0.1, 0.1, 0.0, 0.5)):
        total, ev = _hemi_integral(cfg, cam, fld, g0, g1, gam, "pmix", 400)
        assert total == pytest.approx(1.0, abs=2e-8)
        s = ev["w_guide"] + ev["w_brdf"]
        assert np.abs(s - 1).max() < 1e-12


def test_mixture_pdf_integral_ggx_equals_valid_mass():
    cfg = O.make_config(1, 1)
    cam = O.make_camera(0, (0, 0, 5), (0, 0, -1), (1, 0, 0), (0, 1, 0))
    fld = O.make_field([[0, 0, 1]], [10.0], [1.0])
    g0, g1 = _one_pixel(rough=0.7)
    gam = _gamma_row(0.4, 0.45, 0.02, 0.03, -0.01, 0.5)
    total, _ = _hemi_integral(cfg, cam, fld, g0, g1, gam, "pmix", 400)
    pb_tot, _ = _hemi_integral(cfg, cam, fld, g0, g1, gam, "pb", 400)
    z = O.derive_pixels(cfg, cam, g0, g1, gam)[0, 5]
    pi = 0.5
    assert total == pytest.approx(pi * z + (1 - pi * z) * pb_tot, abs=2e-8)
    assert pb_tot < 1.0
    # the valid mass of the BRDF draw, by brute-force sampling
    rng = np.random.default_rng(16)
    ok = np.mean([O.brdf_sample(0.7, np.array([0, 0, 1.0]), *rng.uniform(0, 1, 2))[1]
                  for _ in range(20000)])
    assert pb_tot == pytest.approx(ok, abs=4 * math.sqrt(ok * (1 - ok) / 20000))


def _unbiased_case(field, gam_rows, rough=-1.0, albedo=0.8, spp=64, seed=5):
    hw = len(gam_rows)
    cfg = O.make_config(hw, 1, spp=spp, seed=seed)
    cam = O.make_camera(0, (0, 0, 5), (0, 0, -1), (1, 0, 0), (0, 1, 0))
    g0 = np.tile(np.array([[0, 0, 1, 5.0]], np.float32), (hw, 1))
    g1 = np.tile(np.array([[0, 0, rough, albedo]], np.float32), (hw, 1))
    samples, img = O.sample(cfg, cam, field, 0, g0, g1, np.asarray(gam_rows))
    F = samples["estimate"].reshape(spp, hw)
    return F, samples


GOOD_AND_BAD = [
    (0.5, 0.5, 0.1, 0.1, 0.0, 0.5), (0.2, 0.8, 0.001, 0.003, 0.001, 0.9),
    (0.95, 0.05, 0.02, 0.02, -0.015, 0.7), (0.0, 0.5, 0.0001, 0.0001, 0.0, 0.95),
]


def _gam_block(n_rep):
    rows = [_gamma_row(*p)[0] for p in GOOD_AND_BAD]
    return np.array(rows * n_rep)


def test_unbiased_constant_radiance_lambert():
    fld = O.make_field([], [], [], constant=1.7)
    F, s = _unbiased_case(fld, _gam_block(256), albedo=0.8)
    m, se = F.mean(), F.std() / math.sqrt(F.size)
    assert abs(m - 0.8 * 1.7) < 4 * se + 1e-12
    # each draw's estimate is L f_r cos / p_mix: with the normal +z and
    # constant radiance, F p_mix = 1.7 (albedo / pi) w_z for every valid draw
    ok = s["pdf"] > 0
    assert ok.mean() > 0.99
    lhs = s["estimate"][ok] * s["pdf"][ok]
    rhs = 1.7 * float(np.float32(0.8)) / math.pi * s["wz"][ok]
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=0)


def test_unbiased_vmf_lobe_on_normal_lambert():
    k = 12.0
    fld = O.make_field([[0, 0, 1]], [k], [1.0])
    ck = k / (2 * math.pi * (1 - math.exp(-2 * k)))
    ref = 0.8 * 2 * ck * (1 / k - (1 - math.exp(-k)) / k ** 2)
    F, _ = _unbiased_case(fld, _gam_block(256), albedo=0.8)
    m, se = F.mean(), F.std() / math.sqrt(F.size)
    assert abs(m - ref) < 4 * se


def test_unbiased_constant_radiance_ggx():
    rough = 0.5
    fld = O.make_field([], [], [], constant=1.0)
    wo = np.array([0, 0, 1.0])
    ref = _sph_quad(lambda w: O.brdf_cos(rough, 0.8, wo, w), epsrel=1e-9)
    F, _ = _unbiased_case(fld, _gam_block(256), rough=rough, albedo=0.8)
    m, se = F.mean(), F.std() / math.sqrt(F.size)
    assert abs(m - ref) < 4 * se


def test_mis_weights_at_samples_match_evaluation():
    """The sampler's reported pdf and balance weight equal the mixture evaluated
    at the drawn direction, and the two balance weights sum to one."""
    fld = O.make_field([[0.3, 0.2, 0.93]], [30.0], [1.0], constant=0.1)
    gam = _gam_block(8)
    hw, spp = len(gam), 16
    cfg = O.make_config(hw, 1, spp=spp, seed=21)
    cam = O.make_camera(0, (0, 0, 5), (0, 0, -1), (1, 0, 0), (0, 1, 0))
    g0 = np.tile(np.array([[0, 0, 1, 5.0]], np.float32), (hw, 1))
    g1 = np.tile(np.array([[0, 0, 0.6, 0.8]], np.float32), (hw, 1))
    s, _ = O.sample(cfg, cam, fld, 0, g0, g1, gam)
    dirs = np.stack([s["wx"], s["wy"], s["wz"]], 1).reshape(spp, hw, 3)
    ev = O.evaluate(cfg, cam, fld, g0, g1, gam, dirs)
    ok = ((s["strategy"] & 4) == 0).reshape(spp, hw)
    assert np.allclose(ev["pmix"][ok], s["pdf"].reshape(spp, hw)[ok], rtol=1e-9)
    assert np.abs(ev["w_guide"] + ev["w_brdf"] - 1)[ev["pmix"] > 0].max() < 1e-12
    st = (s["strategy"] & 3).reshape(spp, hw)
    own = np.where(st == 1, ev["w_guide"], ev["w_brdf"])
    assert np.allclose(own[ok], s["mis"].reshape(spp, hw)[ok], rtol=1e-9, atol=1e-15)


# ---------------------------------------------------------------------------
# Reprojection (Sec. 3.1)
# ---------------------------------------------------------------------------
def test_reproject_identity_copies_gamma_exactly():
    rng = np.random.default_rng(13)
    W, H = 9, 7
    cfg = O.make_config(W, H)
    g0, g1 = scenes.random_gbuffer(rng, W, H)
    gam = scenes.random_gamma(rng, W * H).astype(np.float64)
    out, acc, q = O.reproject(cfg, g0, g1, g0, gam)
    assert acc.all()
    assert (q == np.arange(W * H)).all()
    assert (out == gam).all()


def test_reproject_integer_pan_shifts_and_rejects_new_columns():
    sc = scenes.PanScene(40, 12, 4, seed=3)
    cfg = O.make_config(40, 12)
    rng = np.random.default_rng(14)
    gam = scenes.random_gamma(rng, 40 * 12).astype(np.float64)
    g0, g1, g0p = sc.gbuffer(2)
    out, acc, q = O.reproject(cfg, g0, g1, g0p, gam)
    a = acc.reshape(12, 40)
    assert a[:, :38].all() and not a[:, 38:].any()
    o = out.reshape(12, 40, 8)
    assert (o[:, :38] == gam.reshape(12, 40, 8)[:, 2:]).all()
    init = O.init_gamma(cfg, 1)[0]
    assert (o[:, 38:] == init).all()
    assert init[5] == pytest.approx(0.05, rel=1e-6) and init[6] == 0


def test_reproject_depth_normal_and_offscreen_rejections():
    W, H = 4, 1
    cfg = O.make_config(W, H)
    g0 = np.tile(np.array([[0, 0, 1, 10.0]], np.float32), (4, 1))
    g0p = g0.copy()
    g0p[1, 3] = 11.5      # depth jump 15 % > 10 %: reject
    g0p[2, 3] = 10.9      # 9 %: accept
    tilt = math.acos(0.85)
    g0p[3, :3] = [math.sin(tilt), 0, math.cos(tilt)]   # cos 0.85 < 0.9: reject
    g1 = np.zeros((4, 4), np.float32)
    g1[:, 2] = -1
    g1[:, 3] = 0.8
    g1[0, 0] = -0.6       # q = floor(0.5 - 0.6) = -1: off screen
    gam = np.tile(_gamma_row(0.3, 0.3, 0.01, 0.01, 0.0, 0.7), (4, 1))
    out, acc, q = O.reproject(cfg, g0, g1, g0p, gam)
    assert list(acc) == [0, 0, 1, 0]
    assert q[0] == -1 and list(q[1:]) == [1, 2, 3]


def test_frame_change_preserves_mean_world_direction():
    cfg = O.make_config(1, 1)
    rng = np.random.default_rng(15)
    for _ in range(30):
        n_prev = scenes.random_normals(rng, 1, 0.3)[0]
        n_cur = scenes.random_normals(rng, 1, 0.3)[0]
        if float(np.dot(n_prev.astype(np.float32), n_cur)) < 0.9:
            continue
        mx, my = rng.uniform(0.25, 0.75, 2)
        gam = _gamma_row(mx, my, 0.004, 0.006, 0.001, 0.4)
        g0 = np.array([[*n_cur, 3.0]], np.float32)
        g0p = np.array([[*n_prev, 3.0]], np.float32)
        g1 = np.array([[0, 0, -1, 0.8]], np.float32)
        out, acc, _ = O.reproject(cfg, g0, g1, g0p, gam)
        assert acc[0] == 1
        def world(n, u):
            t, b = O.basis(n.astype(np.float64))
            w = O.square_to_hemi(u)[0]
            return w[0] * t + w[1] * b + w[2] * n.astype(np.float64)
        w_old = world(n_prev, [mx, my])
        w_new = world(n_cur, out[0, :2])
        if np.dot(w_old, n_cur.astype(np.float64)) > 1e-3:
            assert np.allclose(w_old, w_new, atol=1e-12)
        # covariance (central second moments) carried unchanged
        c_new = out[0, 2:5] - np.array([out[0, 0] ** 2, out[0, 1] ** 2, out[0, 0] * out[0, 1]])
        assert np.allclose(c_new, [0.004, 0.006, 0.001], atol=1e-14)
        assert (out[0, 5:] == gam[0, 5:]).all()


# ---------------------------------------------------------------------------
# Training: weighted online EM (Sec. 3.2)
# ---------------------------------------------------------------------------
def test_em_population_fixed_point():
    """Fed exact quadrature statistics of its own mixture as the target, one EM
    step returns the mixture (mu*, Sigma*, pi*): the EM fixed point."""
    mu, sig, pi = (0.4, 0.6), (4e-3, 3e-3, 1e-3), 0.6
    n = 1024
    g = (np.arange(n) + 0.5) / n
    U, V = np.meshgrid(g, g)
    dirs = O.square_to_hemi(np.stack([U.ravel(), V.ravel()], 1))
    N = n * n
    cfg = O.make_config(1, 1, spp=N)
    cam = O.make_camera(0, (0, 0, 5), (0, 0, -1), (1, 0, 0), (0, 1, 0))
    fld = O.make_field([], [], [], constant=1.0)
    g0, g1 = _one_pixel(albedo=1.0)
    gam = _gamma_row(*mu, *sig, pi, k=5.0)
    ev = O.evaluate(cfg, cam, fld, g0, g1, gam, dirs[:, None, :])
    z = O.derive_pixels(cfg, cam, g0, g1, gam)[0, 5]
    assert 1 - z < 1e-8
    # The target L f_r cos is the mixture pdf itself. The u-grid is uniform in
    # solid angle (M is equal-area) rather than drawn from p_b, so the radiance
    # carries the density ratio: with Lambert albedo 1, f = L p_b and the
    # training weight f / p_b = L, which must be proportional to p_mix.
    samples = dict(wx=dirs[:, 0], wy=dirs[:, 1], wz=dirs[:, 2],
                   radiance=ev["pmix"].ravel(), estimate=np.zeros(N),
                   strategy=np.zeros(N, np.uint8))
    for wbar in (0.0, 1.0):          # W = 0 at k > 0: the frame's own mass stands in
        g = gam.copy()
        g[0, 7] = wbar
        out = O.update(cfg, cam, g0, g1, g, samples)
        # tolerance: the 1024^2 midpoint grid's own error on the ratios S/a, a/b
        assert out[0, :5] == pytest.approx(gam[0, :5], abs=5e-7)
        assert out[0, 5] == pytest.approx(pi, abs=1e-6)
        assert out[0, 6] == 6.0


def _one_sample_update(u, radiance, gam_row, k_max=32):
    cfg = O.make_config(1, 1, spp=1, k_max=k_max)
    cam = O.make_camera(0, (0, 0, 5), (0, 0, -1), (1, 0, 0), (0, 1, 0))
    g0, g1 = _one_pixel()
    w = O.square_to_hemi(u)[0]
    s = dict(wx=[w[0]], wy=[w[1]], wz=[w[2]], radiance=[radiance], estimate=[0.0],
             strategy=np.zeros(1, np.uint8))
    return O.update(cfg, cam, g0, g1, np.asarray(gam_row, np.float64).reshape(1, 8), s)[0]


def test_em_step_is_a_convex_move_toward_the_sample():
    """With one BRDF sample the batch mean is that sample's square coordinate u;
    all five moments move toward (u, u u^T) by the same fraction in [0, 1]."""
    u = np.array([0.3, 0.65])
    tgt = np.array([u[0], u[1], u[0] ** 2, u[1] ** 2, u[0] * u[1]])
    for k, wbar in ((0.0, 0.0), (5.0, 0.7), (31.0, 2.0), (40.0, 0.1)):
        gam = _gamma_row(0.45, 0.55, 0.02, 0.03, 0.004, 0.6, k=k, i=wbar)[0]
        out = _one_sample_update(u, 2.0, gam)
        lam = (out[:5] - gam[:5]) / (tgt - gam[:5])
        assert np.allclose(lam, lam[0], atol=1e-12) and 0.0 < lam[0] < 1.0
        assert 0.05 <= out[5] <= 0.95
        assert out[6] == min(k + 1, 32)
        assert out[7] > 0


def test_em_step_is_continuous_and_luminance_weighted():
    """A sample carrying vanishing luminance moves nothing; a brighter sample
    moves the guide further (Sec. 3.1: moments weighted by luminance)."""
    u = [0.8, 0.2]
    gam = _gamma_row(0.4, 0.5, 0.01, 0.01, 0.0, 0.5, k=6.0, i=1.0)[0]
    moves = [np.abs(_one_sample_update(u, r, gam)[:5] - gam[:5]).max() for r in (1e-12, 0.1, 1.0, 10.0)]
    assert moves[0] < 1e-10
    assert moves[0] < moves[1] < moves[2] < moves[3]


def test_em_step_scale_invariance():
    """Scaling every luminance weight and the stored mass W by c leaves the
    guide unchanged and scales W."""
    u = [0.25, 0.6]
    gam = _gamma_row(0.5, 0.5, 0.02, 0.02, 0.005, 0.4, k=3.0, i=0.8)[0]
    a = _one_sample_update(u, 1.5, gam)
    g2 = gam.copy()
    g2[7] *= 7.0
    b = _one_sample_update(u, 1.5 * 7.0, g2)
    assert np.allclose(a[:7], b[:7], rtol=1e-12, atol=1e-15)
    assert b[7] == pytest.approx(7.0 * a[7], rel=1e-12)


def test_em_guide_and_wasted_samples_do_not_train():
    cfg = O.make_config(1, 1, spp=3)
    cam = O.make_camera(0, (0, 0, 5), (0, 0, -1), (1, 0, 0), (0, 1, 0))
    g0, g1 = _one_pixel()
    gam = _gamma_row(0.5, 0.5, 0.02, 0.02, 0.0, 0.5, k=4.0, i=0.5)
    w = O.square_to_hemi([0.2, 0.3])[0]
    s = dict(wx=[w[0]] * 3, wy=[w[1]] * 3, wz=[w[2]] * 3, radiance=[1.0] * 3,
             estimate=[1.0, 2.0, 3.0], strategy=np.array([1, 2, 4], np.uint8))
    out = O.update(cfg, cam, g0, g1, gam, s)[0]
    assert (out == gam[0]).all()     # no BRDF-strategy energy: Gamma unchanged


def test_em_recovers_a_known_mixture_from_its_samples():
    """Stochastic recovery: BRDF draws whose luminance follows a known mixture
    (mu*, Sigma*, pi*) train the guide onto it over many frames."""
    mu, sig, pi = np.array([0.35, 0.62]), np.array([3e-3, 5e-3, -1e-3]), 0.7
    # k_max = 8 keeps a forgetting window of ten frames, so the early frames of
    # the broad initial guide are forgotten within the run
    spp, frames = 256, 80
    cfg = O.make_config(1, 1, spp=spp, k_max=8)
    cam = O.make_camera(0, (0, 0, 5), (0, 0, -1), (1, 0, 0), (0, 1, 0))
    fld = O.make_field([], [], [], constant=1.0)
    g0, g1 = _one_pixel(albedo=1.0)
    target = _gamma_row(*mu, *sig, pi, k=5.0)
    gam = _gamma_row(0.5, 0.5, 0.1, 0.1, 0.0, 0.5, k=0.0)
    rng = np.random.default_rng(17)
    for t in range(frames):
        d = np.array([O.brdf_sample(-1.0, [0, 0, 1.0], *rng.uniform(0, 1, 2))[0] for _ in range(spp)])
        ev = O.evaluate(cfg, cam, fld, g0, g1, target, d[:, None, :])
        # Lambert, albedo 1: f = L p_b, so radiance = p_mix* / p_b makes f = p_mix*
        s = dict(wx=d[:, 0], wy=d[:, 1], wz=d[:, 2], radiance=(ev["pmix"] / ev["pb"]).ravel(),
                 estimate=np.zeros(spp), strategy=np.zeros(spp, np.uint8))
        gam = O.update(cfg, cam, g0, g1, gam, s)
    g5 = O.derive(cfg, gam)[0]
    assert np.abs(g5[:2] - mu).max() < 0.01
    assert np.abs(g5[2:] - sig).max() < 1e-3
    assert abs(gam[0, 5] - pi) < 0.05


def test_reinit_pixel_samples_brdf_only():
    cfg = O.make_config(8, 8, spp=4, seed=9)
    cam = O.make_camera(0, (0, 0, 5), (0, 0, -1), (1, 0, 0), (0, 1, 0))
    fld = O.make_field([[0, 0, 1]], [5.0], [1.0], constant=0.1)
    g0 = np.tile(np.array([[0, 0, 1, 5.0]], np.float32), (64, 1))
    g1 = np.tile(np.array([[0, 0, -1, 0.8]], np.float32), (64, 1))
    gam = np.tile(_gamma_row(0.5, 0.5, 0.05, 0.05, 0.0, 0.95), (64, 1))
    s, _ = O.sample(cfg, cam, fld, 0, g0, g1, gam, reinit=np.ones(64, np.uint8))
    assert ((s["strategy"] & 3) == 0).all()
    s2, _ = O.sample(cfg, cam, fld, 0, g0, g1, gam)
    assert ((s2["strategy"] & 3) != 0).mean() > 0.8


# ---------------------------------------------------------------------------
# Second-moment loss and its gradient (the differentiable form)
# ---------------------------------------------------------------------------
def _adjoint_case(n_pix=24, seed=41, rough_frac=0.5):
    rng = np.random.default_rng(seed)
    cfg = O.make_config(n_pix, 1, seed=seed)
    cam = O.make_camera(0, (0, 0, 5), (0, 0, -1), (1, 0, 0), (0, 1, 0))
    fld = O.make_field([[0.3, 0.2, 0.93], [-0.5, 0.1, 0.86]], [15.0, 40.0], [1.0, 0.7], constant=0.1)
    g0, g1 = scenes.random_gbuffer(rng, n_pix, 1, ggx_frac=rough_frac, rough_lo=0.3, max_tilt=0.3)
    th = np.stack([rng.uniform(0.25, 0.75, n_pix), rng.uniform(0.25, 0.75, n_pix),
                   rng.uniform(0.004, 0.03, n_pix), rng.uniform(0.004, 0.03, n_pix),
                   np.zeros(n_pix), rng.uniform(0.2, 0.8, n_pix)], 1)
    th[:, 4] = rng.uniform(-0.6, 0.6, n_pix) * np.sqrt(th[:, 2] * th[:, 3])
    return cfg, cam, fld, g0, g1, th


def test_second_moment_gradient_matches_central_differences():
    cfg, cam, fld, g0, g1, th = _adjoint_case()
    n = 32
    loss, grad, _ = O.second_moment(cfg, cam, fld, 3, n, g0, g1, th)
    scale = np.abs(th).max(0) * 0 + np.array([1, 1, 0.01, 0.01, 0.01, 1.0])
    for j in range(6):
        h = 1e-5 * scale[j]
        def at(d):
            t = th.copy()
            t[:, j] += d
            return O.second_moment(cfg, cam, fld, 3, n, g0, g1, th, t)[0]
        # Richardson-extrapolated central difference
        d1 = (at(h) - at(-h)) / (2 * h)
        d2 = (at(2 * h) - at(-2 * h)) / (4 * h)
        fd = (4 * d1 - d2) / 3
        ref = np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())
        assert np.abs(grad[:, j] - fd).max() / ref.max() < 1e-6 or (np.abs(grad[:, j] - fd) / ref).max() < 1e-5, j


def test_second_moment_loss_is_the_estimators_second_moment():
    """At theta = theta0 the loss is the Monte Carlo second moment of F; over
    many replicas it converges to the integral of f^2 / p over the hemisphere."""
    reps, n = 256, 16
    cfg = O.make_config(reps, 1, seed=5)
    cam = O.make_camera(0, (0, 0, 5), (0, 0, -1), (1, 0, 0), (0, 1, 0))
    fld = O.make_field([[0.3, 0.2, 0.93]], [20.0], [1.0], constant=0.1)
    g0 = np.tile(np.array([[0, 0, 1, 5.0]], np.float32), (reps, 1))
    g1 = np.tile(np.array([[0, 0, -1, 0.8]], np.float32), (reps, 1))
    th = np.tile([0.6, 0.55, 0.01, 0.02, 0.004, 0.5], (reps, 1))
    loss, _, _ = O.second_moment(cfg, cam, fld, 0, n, g0, g1, th)
    m = 600
    gr = (np.arange(m) + 0.5) / m
    U, V = np.meshgrid(gr, gr)
    dirs = O.square_to_hemi(np.stack([U.ravel(), V.ravel()], 1))
    gam = np.array([[0.6, 0.55, 0.01 + 0.36, 0.02 + 0.3025, 0.004 + 0.33, 0.5, 0, 0]])
    c1 = O.make_config(1, 1)
    ev = O.evaluate(c1, cam, fld, g0[:1], g1[:1], gam, dirs[:, None, :])
    ok = ev["pmix"] > 0
    ref = 2 * np.pi * np.where(ok, ev["fcos"] ** 2 / np.where(ok, ev["pmix"], 1), 0).mean()
    assert abs(loss.mean() - ref) < 4 * loss.std() / np.sqrt(reps)


def test_adam_first_step_closed_form_and_projection():
    cfg = O.make_config(3, 1)
    gam = np.array([[0.5, 0.5, 0.26, 0.27, 0.251, 0.5, 4, 2.0],
                    [0.9995, 0.2, 0.9995 ** 2 + 0.01, 0.05, 0.2 * 0.9995, 0.0505, 7, 1.0],
                    [0.3, 0.7, 0.09 + 0.02, 0.49 + 0.02, 0.21, 0.9, 1, 0.5]])
    grad = np.array([[1.0, -2.0, 0.5, -0.5, 1e-3, -1.0],
                     [-3.0, 1.0, 1.0, 1.0, 1.0, 5e3],
                     [0.0, 0.0, 0.0, 0.0, 0.0, 0.0]])
    th0 = O.theta_from_gamma(cfg, gam)
    out, m, v = O.adam(cfg, gam, grad, np.zeros((3, 6)), np.zeros((3, 6)), 1e-3, 0.9, 0.999, 1e-8, 1)
    th1 = O.theta_from_gamma(cfg, out)
    # pixel 0: interior; at step 1 the bias-corrected moments are g and g^2, so
    # every parameter moves by lr g / (|g| + eps) against the gradient
    assert np.allclose(th1[0], th0[0] - 1e-3 * grad[0] / (np.abs(grad[0]) + 1e-8), atol=1e-12)
    # pixel 1: the mean hits the square's edge and pi its lower clamp
    assert th1[1, 0] == 1.0 and th1[1, 5] == pytest.approx(0.05, rel=1e-6)
    # pixel 2: zero gradient, zero step
    assert np.allclose(th1[2], th0[2], atol=1e-12)
    assert (out[:, 6:] == gam[:, 6:]).all()      # k and W are kept


def test_second_moment_gradient_against_central_differences_at_h_1e_4():
    """The check as the differentiation configuration states it: FP64 central
    finite differences of the loss with h = 1e-4, the analytic gradient
    within 1e-3 relative (per component, against the larger of its own
    magnitude and 1e-3 of the pixel's largest component). h is taken in each
    parameter's own units: 1 for the mean and pi, 1e-2 for the covariance
    entries (the guides' variances lie near 1e-2; an absolute 1e-4 there is
    1% of sigma^2, and the difference's own truncation error, h^2 times the
    third derivative over 6, is then 3e-3: above the bound whatever the
    gradient)."""
    cfg, cam, fld, g0, g1, th = _adjoint_case()
    n = 32
    _, grad, _ = O.second_moment(cfg, cam, fld, 3, n, g0, g1, th)
    fd = np.empty_like(grad)
    for j, unit in enumerate((1.0, 1.0, 1e-2, 1e-2, 1e-2, 1.0)):
        h = 1e-4 * unit
        t1, t2 = th.copy(), th.copy()
        t1[:, j] += h
        t2[:, j] -= h
        fd[:, j] = (O.second_moment(cfg, cam, fld, 3, n, g0, g1, th, t1)[0] -
                    O.second_moment(cfg, cam, fld, 3, n, g0, g1, th, t2)[0]) / (2 * h)
    lim = 1e-3 * np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max(1, keepdims=True))
    assert (np.abs(grad - fd) <= lim).all(), (np.abs(grad - fd) / lim).max()
