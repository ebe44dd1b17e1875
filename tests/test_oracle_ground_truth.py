"""Pins of the oracle's ground truth I(p) = int L f_r cos dw (Eq. 1), of its
camera rays and of the radiance field's occlusion mask.

Each is checked against something other than itself: closed forms (constant
radiance, a von Mises-Fisher lobe on the normal and one far from the
horizon), an independent quadrature (the GGX directional albedo over half
vectors, a masked field on a midpoint grid of the square), the mean of the
pass's own unbiased estimator, and the geometry the synthetic scenes were
built from (the panned heightfield, the orbit's ground and quads).
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from paper_2112_09728_gb300 import scenes

F32 = lambda v: float(np.float32(v))


def _pixel(normal=(0.0, 0.0, 1.0), rough=-1.0, albedo=0.8, depth=5.0):
    n = np.asarray(normal, np.float64)
    n /= np.linalg.norm(n)
    g0 = np.array([[*n, depth]], np.float32)
    g1 = np.array([[0.0, 0.0, rough, albedo]], np.float32)
    return g0, g1


def _view_camera(theta_deg, phi_deg=0.0):
    """Orthographic camera whose rays arrive at angle theta from +z (w_o at theta)."""
    th, ph = math.radians(theta_deg), math.radians(phi_deg)
    wo = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    fwd = -wo
    right = np.cross(fwd, [0.0, 0.0, 1.0]) if abs(wo[2]) < 0.999 else np.array([1.0, 0.0, 0.0])
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    return O.make_camera(0, 5.0 * wo, fwd, right, up, pixel_size=1e-9), wo


def _gt(fld, g0, g1, cam=None, tol=1e-10, **cfg_kw):
    cfg = O.make_config(1, 1, **cfg_kw)
    cam = cam or O.make_camera(0, (0, 0, 5), (0, 0, -1), (1, 0, 0), (0, 1, 0))
    I, err = O.ground_truth(cfg, cam, fld, g0, g1, [0], [0], tol_rel=tol, with_error=True)
    return I[0], err[0]


# ---------------------------------------------------------------------------
# Closed forms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("normal", [(0, 0, 1), (0.3, -0.2, 0.9), (0.7, 0.1, 0.4)])
def test_constant_radiance_lambert_gives_albedo_times_radiance(normal):
    fld = O.make_field([], [], [], constant=1.7)
    cam, _ = _view_camera(25.0, 40.0)
    I, _ = _gt(fld, *_pixel(normal, albedo=0.6), cam=cam)
    assert I == pytest.approx(F32(0.6) * 1.7, rel=1e-12)


def _vmf_c(k):
    return k / (2 * math.pi * (1 - math.exp(-2 * k)))


@pytest.mark.parametrize("kappa", [5.0, 80.0, 500.0])
def test_vmf_lobe_on_the_normal_closed_form(kappa):
    # rho/pi int C e^{k(z-1)} z dw = 2 rho C [1/k - (1 - e^-k)/k^2]
    n = np.array([0.2, 0.1, 0.97])
    n /= np.linalg.norm(n)
    n32 = np.asarray(n, np.float32).astype(np.float64)
    fld = O.make_field([n32 / np.linalg.norm(n32)], [kappa], [1.3])
    I, _ = _gt(fld, *_pixel(n32, albedo=0.8))
    ref = 1.3 * F32(0.8) * 2 * _vmf_c(kappa) * (1 / kappa - (1 - math.exp(-kappa)) / kappa ** 2)
    # the lobe axis and the binary32 normal agree to ~1e-8
    assert I == pytest.approx(ref, rel=1e-6 if kappa == 500 else 1e-7)


@pytest.mark.parametrize("kappa,angle", [(200.0, 30.0), (200.0, 45.0), (50.0, 20.0)])
def test_vmf_lobe_away_from_the_horizon_closed_form(kappa, angle):
    # over the whole sphere int vMF(w) (n.w) dw = A(k) n.d with A(k) = coth k - 1/k
    # (the lobe's mean resultant length); the part below the horizon is below
    # e^{-k (1 - sin(angle))} < 1e-14 here
    a = math.radians(angle)
    d = [math.sin(a), 0.0, math.cos(a)]
    fld = O.make_field([d], [kappa], [1.0])
    I, _ = _gt(fld, *_pixel(albedo=0.8))
    ref = F32(0.8) / math.pi * (1 / math.tanh(kappa) - 1 / kappa) * math.cos(a)
    assert I == pytest.approx(ref, rel=1e-10)


def _ggx_albedo_half_vectors(rough, f0, theta_o):
    """Directional albedo (per unit albedo) of the GGX lobe by quadrature over
    half vectors h: int F D G1(i) G1(o) (o.h)/cos_o dw_h, w_i = 2 (o.h) h - o,
    over the h whose reflection stays above the horizon (the change of
    variables dw_i = 4 (o.h) dw_h)."""
    a = max(rough * rough, 1e-4)
    a2 = a * a
    o = np.array([math.sin(theta_o), 0.0, math.cos(theta_o)])
    D = lambda c: a2 / (math.pi * (c * c * (a2 - 1) + 1) ** 2)
    G1 = lambda c: 2 * c / (c + math.sqrt(a2 + (1 - a2) * c * c))

    def f(ph, th):
        h = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        oh = float(o @ h)
        if oh <= 0:
            return 0.0
        wi_z = 2 * oh * h[2] - o[2]
        if wi_z <= 0:
            return 0.0
        fr = f0 + (1 - f0) * (1 - oh) ** 5
        return fr * D(h[2]) * G1(wi_z) * G1(o[2]) * oh / o[2] * math.sin(th)

    pts = [a * k for k in (1, 2, 4, 8) if a * k < math.pi / 2]
    v, _ = integrate.nquad(f, [[0, 2 * math.pi], [0, math.pi / 2]],
                           opts=[{"epsabs": 1e-13, "epsrel": 1e-11, "limit": 200},
                                 {"epsabs": 1e-13, "epsrel": 1e-11, "limit": 200, "points": pts}])
    return v


@pytest.mark.parametrize("rough,f0,theta", [(0.6, 1.0, 0.0), (0.4, 1.0, 40.0), (0.15, 1.0, 40.0),
                                            (0.4, 0.3, 70.0)])
def test_ggx_constant_radiance_equals_albedo_over_half_vectors(rough, f0, theta):
    fld = O.make_field([], [], [], constant=1.0)
    cam, _ = _view_camera(theta)
    I, _ = _gt(fld, *_pixel(rough=rough, albedo=0.9), cam=cam, ggx_f0=f0)
    ref = F32(0.9) * _ggx_albedo_half_vectors(F32(rough), F32(f0), math.radians(theta))
    assert I == pytest.approx(ref, rel=2e-9)


@pytest.mark.parametrize("rough", [0.05, 0.02])
def test_ggx_sharp_lobe_at_normal_incidence(rough):
    # one-dimensional in theta_h at normal incidence (w_i at 2 theta_h)
    r = F32(rough)
    a = max(r * r, 1e-4)
    a2 = a * a
    D = lambda c: a2 / (math.pi * (c * c * (a2 - 1) + 1) ** 2)
    G1 = lambda c: 2 * c / (c + math.sqrt(a2 + (1 - a2) * c * c))
    f = lambda th: D(math.cos(th)) * G1(math.cos(2 * th)) * math.cos(th) * math.sin(th)
    v, _ = integrate.quad(f, 0, math.pi / 4, epsabs=0, epsrel=1e-12, limit=500,
                          points=[a * k for k in (0.5, 1, 2, 4, 8, 16) if a * k < math.pi / 4])
    fld = O.make_field([], [], [], constant=1.0)
    I, err = _gt(fld, *_pixel(rough=rough, albedo=0.8), tol=1e-9)
    assert I == pytest.approx(F32(0.8) * 2 * math.pi * v, rel=3e-8)
    assert err < 1e-8


# ---------------------------------------------------------------------------
# Independent quadrature and the estimator
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("rough", [-1.0, 0.6])
def test_masked_field_against_a_midpoint_grid_on_the_square(rough):
    """A masked two-lobe field: the cubature against 2 pi times the mean over a
    midpoint grid of the square mapped by M (equal area), Richardson-extrapolated."""
    fld = O.make_field([[0.3, 0.2, 0.93], [-0.5, 0.1, 0.86]], [20.0, 35.0], [1.0, 0.7], constant=0.05,
                       mask=(0.21, 0.17, 0.5))
    # the normal +z is exactly unit in binary32, so the evaluator's round trip
    # of each direction through the local frame is exact; the view is oblique
    g0, g1 = _pixel((0.0, 0.0, 1.0), rough=rough, albedo=0.7, depth=3.0)
    cfg = O.make_config(1, 1)
    cam, _ = _view_camera(35.0, 120.0)
    I = O.ground_truth(cfg, cam, fld, g0, g1, [0], [0], tol_rel=1e-11)[0]
    nn = g0[0, :3].astype(np.float64)
    t, b = O.basis(nn)
    gam = O.init_gamma(cfg, 1)
    vals = []
    for m in (700, 1400):
        gr = (np.arange(m) + 0.5) / m
        U, V = np.meshgrid(gr, gr)
        wl = O.square_to_hemi(np.stack([U.ravel(), V.ravel()], 1))
        ww = wl[:, :1] * t + wl[:, 1:2] * b + wl[:, 2:3] * nn
        # L f_r cos at each direction (the pieces the estimator uses)
        f = O.evaluate(cfg, cam, fld, g0, g1, gam, ww[:, None, :])["fcos"]
        vals.append(2 * np.pi * f.mean())
    ref = (4 * vals[1] - vals[0]) / 3
    assert I == pytest.approx(ref, rel=2e-7)
    assert abs(vals[1] - ref) > 10 * abs(I - ref)     # the grid's own error is far larger


def test_ground_truth_is_the_mean_of_the_pass_estimator():
    """On a 16 x 2 screen of the pan workload's scene (heightfield normals,
    Lambert and GGX texels, the masked four-lobe field), the oracle's unbiased
    estimator averaged over many draws from the initial guide lands on I(p)
    within 4.5 standard errors at every pixel."""
    wl = scenes.workload_pan(16, 2, frames=2)
    par, fld, sc = wl["params"], wl["field"], wl["scene"]
    g0, g1, _ = sc.gbuffer(1)
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    of = O.make_field(f32(fld.dirs), f32(fld.kappas), f32(fld.amps), F32(fld.constant), [F32(m) for m in fld.mask])
    c = sc.camera(1)
    cam = O.make_camera(c.kind, c.origin, c.fwd, c.right, c.up, c.pixel_size)
    cfg = O.make_config(16, 2, spp=5000, seed=9)
    xs, ys = np.arange(32) % 16, np.arange(32) // 16
    I = O.ground_truth(cfg, cam, of, g0, g1, xs, ys, tol_rel=1e-9)
    gam = np.tile(O.init_gamma(cfg, 1, pi=0.5)[0], (32, 1))
    s, _ = O.sample(cfg, cam, of, 0, g0, g1, gam)
    F = s["estimate"].reshape(cfg.spp, 32)
    se = F.std(0) / math.sqrt(cfg.spp)
    assert (np.abs(F.mean(0) - I) < 4.5 * se + 1e-12).all(), np.max(np.abs(F.mean(0) - I) / se)
    assert (g1[:, 2] >= 0).any() and (g1[:, 2] < 0).any()


def test_transparent_pixel_and_view_from_below():
    fld = O.make_field([[0.3, 0.2, 0.93]], [15.0], [1.0], constant=0.2, mask=(0.3, 0.2, 0.5))
    cam, _ = _view_camera(35.0, 10.0)
    cfg = O.make_config(1, 1, spp=4000, seed=3, transparent=1)
    g0, g1 = _pixel((0.1, 0.0, 1.0), rough=-2.0, albedo=0.9)
    I = O.ground_truth(cfg, cam, fld, g0, g1, [0], [0])[0]
    s, _ = O.sample(cfg, cam, fld, 0, g0, g1, O.init_gamma(cfg, 1))
    F = s["estimate"]
    assert abs(F.mean() - I) < 4.5 * F.std() / math.sqrt(len(F))
    assert I > 0
    # seen from below the surface nothing is reflected: I = 0
    for rough in (-1.0, 0.3, -2.0):
        g0b, g1b = _pixel((0.0, 0.0, -1.0), rough=rough)
        assert O.ground_truth(cfg, O.make_camera(0, (0, 0, 5), (0, 0, -1), (1, 0, 0), (0, 1, 0)), fld,
                              g0b, g1b, [0], [0])[0] == 0.0


def test_coloured_field_integrates_each_channel():
    """Each channel of a coloured field's ground truth is the ground truth of
    the monochrome field carrying that channel's amplitudes."""
    dirs = [[0.3, 0.2, 0.93], [-0.4, 0.3, 0.87]]
    rgb = [[1.0, 0.5, 0.2], [0.1, 0.9, 0.4]]
    const = (0.05, 0.1, 0.02)
    fld = O.make_field(dirs, [30.0, 60.0], [1.0, 1.0], mask=(0.2, 0.3, 0.5), rgb=rgb, constant_rgb=const)
    g0, g1 = _pixel((0.1, 0.05, 1.0), rough=0.35, albedo=0.8)
    cfg = O.make_config(1, 1)
    cam = O.make_camera(0, (0.4, 0.7, 5), (0, 0, -1), (1, 0, 0), (0, 1, 0))
    I = O.ground_truth(cfg, cam, fld, g0, g1, [0], [0], tol_rel=1e-10)[0]
    for c in range(3):
        mono = O.make_field(dirs, [30.0, 60.0], [rgb[0][c], rgb[1][c]], constant=const[c], mask=(0.2, 0.3, 0.5))
        assert I[c] == pytest.approx(O.ground_truth(cfg, cam, mono, g0, g1, [0], [0], tol_rel=1e-10)[0], rel=1e-8)


# ---------------------------------------------------------------------------
# Camera rays
# ---------------------------------------------------------------------------
def test_orthographic_rays_land_on_the_panned_heightfield():
    """Pan workload: pixel (x, y) of frame t sees world texel (x + 2t, y); the
    shading point origin + depth * dir is that texel's centre on the fBm
    heightfield."""
    W, H = 96, 40
    sc = scenes.PanScene(W, H, 12, scenes.SEED_BASE + 2)
    hf = scenes.Heightfield(scenes.SEED_BASE + 2)
    rng = np.random.default_rng(1)
    for t in (0, 7):
        g0, _, _ = sc.gbuffer(t)
        c = sc.camera(t)
        cam = O.make_camera(c.kind, c.origin, c.fwd, c.right, c.up, c.pixel_size)
        for _ in range(20):
            x, y = int(rng.integers(W)), int(rng.integers(H))
            o, d = O.camera_ray(cam, W, H, x, y)
            p = o + float(g0[y * W + x, 3]) * d
            xw, yw = x + 2 * t + 0.5, y + 0.5
            h, _, _ = hf.eval(np.array([xw]), np.array([yw]))
            assert p[0] == pytest.approx(xw, abs=1e-12) and p[1] == pytest.approx(yw, abs=1e-12)
            assert p[2] == pytest.approx(h[0], abs=1e-5)          # depth stored in binary32
            assert np.allclose(d, [0, 0, -1])


def test_pinhole_rays_land_on_the_orbit_scene():
    """Orbit workload at a small size: origin + depth * dir is the generator's
    own ray-cast hit (on the ground plane z = 0 or on a quad) for every pixel."""
    W, H = 48, 27
    sc = scenes.QuadScene(W, H, scenes.SEED_BASE + 5)
    for t in (0, 30):
        g0, _, _ = sc.gbuffer(t)
        P, _, depth, _ = sc._cast(scenes._NP(), t)
        P = P.reshape(-1, 3)
        c = sc.camera(t)
        cam = O.make_camera(c.kind, c.origin, c.fwd, c.right, c.up, tan_half_fov=c.tan_half_fov)
        fin = np.isfinite(depth.reshape(-1)) & (depth.reshape(-1) < 999)
        assert fin.mean() > 0.5
        for i in np.nonzero(fin)[0]:
            o, d = O.camera_ray(cam, W, H, i % W, i // W)
            p = o + float(g0[i, 3]) * d
            assert np.allclose(p, P[i], atol=2e-6 * float(g0[i, 3]) + 1e-9), (i, p, P[i])
        ground = fin & (np.abs(P[:, 2]) < 1e-9)
        assert ground.mean() > 0.2


def test_pinhole_centre_ray_and_horizontal_field_of_view():
    """A 60 degree horizontal field of view (the orbit workload's): the centre
    pixel of an odd screen looks along fwd, the outermost pixel columns at
    atan(tan 30 deg (1 - 1/W)), row 0 is the top of the image, column 0 the
    left."""
    W, H = 41, 23
    tan_v = math.tan(math.radians(30.0)) * H / W
    fwd, right, up = np.array([0.6, 0.8, 0.0]), np.array([0.8, -0.6, 0.0]), np.array([0.0, 0.0, 1.0])
    cam = O.make_camera(1, (1, 2, 3), fwd, right, up, tan_half_fov=tan_v)
    _, d = O.camera_ray(cam, W, H, W // 2, H // 2)
    assert np.allclose(d, fwd, atol=1e-15)
    for x, sgn in ((W - 1, 1.0), (0, -1.0)):
        _, d = O.camera_ray(cam, W, H, x, H // 2)
        ang = math.atan2(d @ right, d @ fwd)
        assert ang == pytest.approx(sgn * math.atan(math.tan(math.radians(30.0)) * (1 - 1 / W)), rel=1e-13)
    _, top = O.camera_ray(cam, W, H, W // 2, 0)
    assert top @ up > 0
    _, bot = O.camera_ray(cam, W, H, W // 2, H - 1)
    assert bot @ up < 0


# ---------------------------------------------------------------------------
# The occlusion mask of the radiance field
# ---------------------------------------------------------------------------
def test_occlusion_mask_values_and_range():
    """L = amp vMF(w) m(x, w) + c with m = 1/2 + 1/2 sin(2 pi (f1 x + g w_x))
    cos(2 pi (f2 y + g w_y)): at w on the lobe's axis vMF = C_k, and the mask
    takes 1, 0 and 1/2 where the sine and cosine take known values; elsewhere
    it stays in [0, 1]."""
    k, amp, c = 10.0, 1.5, 0.07
    f1, f2, g = 1 / 97.0, 1 / 131.0, 0.5
    d = np.array([0.3, 0.2, math.sqrt(1 - 0.13)])
    fld = O.make_field([d], [k], [amp], constant=c, mask=(f1, f2, g))
    peak = amp * _vmf_c(k)
    y0 = -g * d[1] / f2                                   # cos(...) = 1
    for arg, m in ((0.25, 1.0), (0.75, 0.0), (0.0, 0.5), (0.5, 0.5)):
        x = (arg - g * d[0]) / f1
        assert O.radiance(fld, [x, y0, 0.0], d) == pytest.approx(peak * m + c, rel=1e-12, abs=1e-14)
    yq = (0.25 - g * d[1]) / f2                           # cos(...) = 0: m = 1/2 whatever the sine
    assert O.radiance(fld, [3.7, yq, 0.0], d) == pytest.approx(0.5 * peak + c, rel=1e-12)
    rng = np.random.default_rng(2)
    for _ in range(200):
        x = rng.uniform(-500, 500, 3)
        w = rng.normal(size=3)
        w /= np.linalg.norm(w)
        v = _vmf_c(k) * math.exp(k * (w @ d - 1))
        m = (O.radiance(fld, x, w) - c) / (amp * v)
        assert -1e-12 <= m <= 1 + 1e-12
