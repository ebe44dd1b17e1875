"""Pins of the oracle's transparent surface and GGX Fresnel term (CPU).

* Dielectric Fresnel against the textbook sine/tangent form of the Fresnel
  equations, with its closed forms at normal and grazing incidence.
* The refracted direction obeys Snell's law, lies in the plane of the view
  direction and the normal, and is a unit vector; the reflection is the mirror.
* A transparent pixel's estimate: under a constant field every sample is
  exactly albedo * L0; under a lobe field the mean over many frames is
  albedo (F L(w_r) + (1 - F) L(w_t)) (a two-outcome binomial check); it never
  trains its guide.
* Schlick's term: F0 = 1 leaves the GGX lobe unchanged, F = F0 at normal
  incidence, and the Fresnel-weighted lobe stays consistent with the BRDF
  sampler (quadrature of f against the mean of f / p over draws).
"""
import math

import numpy as np

import oracle as O
from paper_2112_09728_gb300 import scenes

from _pg import ocam

N_IOR = 1.5


def _fresnel_sin_tan(ti):
    tt = math.asin(math.sin(ti) / N_IOR)
    if ti == 0.0:
        r = (N_IOR - 1) / (N_IOR + 1)
        return r * r
    rs = -math.sin(ti - tt) / math.sin(ti + tt)
    rp = math.tan(ti - tt) / math.tan(ti + tt)
    return 0.5 * (rs * rs + rp * rp)


def test_dielectric_fresnel_against_the_sine_tangent_form():
    assert abs(O.dielectric_fresnel(1.0) - 0.04) < 1e-15
    assert abs(O.dielectric_fresnel(1e-9) - 1.0) < 1e-6
    prev = 0.0
    for ti in np.linspace(0.0, math.pi / 2 - 1e-3, 200):
        f = O.dielectric_fresnel(math.cos(ti))
        assert abs(f - _fresnel_sin_tan(ti)) < 1e-12
        assert f >= prev - 1e-15          # external reflection grows with the angle
        prev = f


def test_refraction_and_reflection_directions():
    rng = np.random.default_rng(3)
    for _ in range(200):
        ti, ph = rng.uniform(0, 1.5), rng.uniform(0, 2 * math.pi)
        wo = np.array([math.sin(ti) * math.cos(ph), math.sin(ti) * math.sin(ph), math.cos(ti)])
        f = O.dielectric_fresnel(wo[2])
        wr, ok_r = O.brdf_sample(-2.0, wo, max(f - 1e-3, 0.0), 0.5)
        wt, ok_t = O.brdf_sample(-2.0, wo, min(f + 1e-3, 0.999), 0.5)
        assert ok_r and ok_t
        assert np.allclose(wr, [-wo[0], -wo[1], wo[2]], atol=1e-15)
        assert abs(np.linalg.norm(wt) - 1) < 1e-12 and wt[2] < 0
        sin_t = math.hypot(wt[0], wt[1])
        assert abs(sin_t - math.sin(ti) / N_IOR) < 1e-12          # Snell
        assert abs(wt[0] * wo[1] - wt[1] * wo[0]) < 1e-12          # in the plane of wo and n
        assert wt[0] * wo[0] + wt[1] * wo[1] <= 1e-15               # on the far side of the normal
    wo = np.array([0.3, 0.0, -0.95])
    wo /= np.linalg.norm(wo)
    _, ok = O.brdf_sample(-2.0, wo, 0.5, 0.5)
    assert not ok                          # viewed from below: a wasted draw


def _glass(W, H, albedo=0.7):
    g0 = np.zeros((W * H, 4), np.float32)
    g0[:, 2] = 1.0
    g0[:, 3] = 3.0
    g1 = np.zeros((W * H, 4), np.float32)
    g1[:, 2] = -2.0
    g1[:, 3] = albedo
    return g0, g1


def test_transparent_pixel_under_constant_field_is_exact_and_never_trains():
    W, H = 8, 6
    g0, g1 = _glass(W, H)
    cfg = O.make_config(W, H, spp=3, seed=9, transparent=1)
    cam = ocam(scenes.top_down_camera(pixel_size=0.2))
    fld = O.make_field(np.zeros((0, 3)), np.zeros(0), np.zeros(0), 0.6)
    rng = np.random.default_rng(0)
    gam = O.init_gamma(cfg, W * H)
    gam[:, 6] = rng.integers(0, 30, W * H)
    gam[:, 7] = rng.uniform(0.1, 2.0, W * H)
    out, acc, s, img = O.frame(cfg, cam, fld, 2, g0, g1, g0, gam)
    a32 = float(np.float32(0.7))
    assert (acc == 1).all()
    assert (s["strategy"] == 3).all() and (s["mis"] == 1.0).all() and (s["pdf"] == 0.0).all()
    assert np.allclose(s["estimate"], a32 * 0.6, rtol=1e-14, atol=0)
    assert np.allclose(img, a32 * 0.6, rtol=1e-14, atol=0)
    assert np.array_equal(out, gam)         # no BRDF-strategy samples: the guide is kept
    # without the transparent material enabled the code is Lambertian
    g1l = g1.copy()
    g1l[:, 2] = -1.0
    off = O.make_config(W, H, spp=3, seed=9)
    a = O.frame(off, cam, fld, 2, g0, g1, g0, gam)
    b = O.frame(off, cam, fld, 2, g0, g1l, g0, gam)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[3], b[3])


def test_transparent_pixel_mean_is_the_fresnel_mix_of_its_two_deltas():
    W, H, frames = 16, 16, 40
    g0, g1 = _glass(W, H, albedo=0.9)
    cfg = O.make_config(W, H, spp=2, seed=21, transparent=1)
    cam = scenes.top_down_camera(pixel_size=0.2)
    d = np.array([[0.3, 0.2, -0.93]])
    d /= np.linalg.norm(d)                  # a lobe below the surface: seen through the glass
    fld = O.make_field(d, np.array([4.0]), np.array([1.0]), 0.05)
    gam = O.init_gamma(cfg, W * H)
    tot = np.zeros(W * H)
    for f in range(frames):
        _, _, _, img = O.frame(cfg, ocam(cam), fld, f, g0, g1, g0, gam)
        tot += img
    mean = tot / frames
    # the view direction of a top-down orthographic camera is +z in every pixel
    wo = np.array([0.0, 0.0, 1.0])
    fr = O.dielectric_fresnel(1.0)
    L = lambda w: O.radiance(fld, np.zeros(3), w)
    w_r, w_t = np.array([0.0, 0.0, 1.0]), np.array([0.0, 0.0, -1.0])
    a = float(np.float32(0.9))
    want = a * (fr * L(w_r) + (1 - fr) * L(w_t))
    # each pixel mean averages 2 * frames two-outcome draws
    sd = a * abs(L(w_r) - L(w_t)) * math.sqrt(fr * (1 - fr) / (2 * frames * W * H))
    assert abs(mean.mean() - want) < 5 * sd + 1e-12


def test_schlick_fresnel_limits_and_consistency_with_the_sampler():
    rng = np.random.default_rng(5)
    for _ in range(20):
        rough = rng.uniform(0.1, 1.0)
        wo = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), 1.0])
        wo /= np.linalg.norm(wo)
        wi = np.array([rng.uniform(-0.6, 0.6), rng.uniform(-0.6, 0.6), 1.0])
        wi /= np.linalg.norm(wi)
        assert O.brdf_cos_f0(rough, 0.8, 1.0, wo, wi) == O.brdf_cos(rough, 0.8, wo, wi)
    n = np.array([0.0, 0.0, 1.0])
    assert abs(O.brdf_cos_f0(0.5, 1.0, 0.04, n, n) / O.brdf_cos(0.5, 1.0, n, n) - 0.04) < 1e-14
    # quadrature of f cos over the hemisphere against the mean of f / p over the sampler's draws
    for rough, ti in ((0.4, 0.3), (0.8, 1.0)):
        wo = np.array([math.sin(ti), 0.0, math.cos(ti)])
        nt, npp = 400, 400
        quad = 0.0
        for a in (np.arange(nt) + 0.5) / nt * (math.pi / 2):
            for b in (np.arange(npp) + 0.5) / npp * (2 * math.pi):
                w = np.array([math.sin(a) * math.cos(b), math.sin(a) * math.sin(b), math.cos(a)])
                quad += O.brdf_cos_f0(rough, 1.0, 0.04, wo, w) * math.sin(a)
        quad *= (math.pi / 2 / nt) * (2 * math.pi / npp)
        m, cnt = 0.0, 0
        k = 300
        for x1 in (np.arange(k) + 0.5) / k:
            for x2 in (np.arange(k) + 0.5) / k:
                w, ok = O.brdf_sample(rough, wo, x1, x2)
                cnt += 1
                if ok:
                    m += O.brdf_cos_f0(rough, 1.0, 0.04, wo, w) / O.brdf_pdf(rough, wo, w)
        assert abs(m / cnt - quad) < 5e-3 * quad, (rough, ti, m / cnt, quad)
