"""The oracle's per-pixel frame (oracle.frame_pixels, the reference of the
full-size parity tests) equals its whole-frame computation (oracle.frame)
on the same pixels, exactly: the same steps run for each pixel in the same
order. The case covers reprojection with rejections, both materials plus the
transparent one, the Fresnel term, a coloured field and two samples."""
import numpy as np

import oracle as O
from paper_2112_09728_gb300 import scenes

from _pg import ocam, ofld


def test_frame_pixels_equals_the_whole_frame():
    W, H, spp, frame = 40, 24, 2, 3
    rng = np.random.default_rng(5)
    g0, g1 = scenes.random_gbuffer(rng, W, H, rough_lo=0.05, glass_frac=0.1)
    moved = rng.random(W * H) < 0.4                                          # the rest keep their pixel
    g1[moved, 0:2] = rng.uniform(-2.5, 2.5, (moved.sum(), 2)).astype(np.float32)   # some land off the screen
    g0p = g0.copy()
    g0p[rng.random(W * H) < 0.2, 3] *= 1.5                                   # depth changes: rejections
    cfg = O.make_config(W, H, spp=spp, seed=77, transparent=1, ggx_f0=0.3)
    cam = ocam(scenes.top_down_camera(pixel_size=0.3))
    fld = ofld(scenes.coloured(scenes.masked_lobe_field(3, n_lobes=3, kappa_hi=200.0, constant=0.05), 4))
    row = O.init_gamma(cfg, 1, pi=0.5)[0]
    row[6], row[7] = 5.0, 0.7                                               # a trained history
    gam = np.tile(row, (W * H, 1))
    out, acc, s, img = O.frame(cfg, cam, fld, frame, g0, g1, g0p, gam)
    assert 0.1 < (acc == 0).mean() < 0.9
    idx = rng.choice(W * H, 150, replace=False)
    xs, ys = idx % W, idx // W
    g, im, margin = O.frame_pixels(cfg, cam, fld, frame, g0, g1, g0p, row, xs, ys)
    assert np.array_equal(g, out[idx])
    assert np.array_equal(im, img.reshape(3, -1)[:, idx].T)
    assert np.array_equal(margin, s["margin"].reshape(spp, -1)[:, idx].min(0))


def test_frame_pixels_from_a_whole_previous_gamma_equals_the_whole_frame():
    """With a different previous Gamma at every pixel (gathered at each pixel's
    reprojected pixel), the per-pixel frame equals the whole-frame oracle
    exactly, accept flags included: the state-synced form of the full-size
    parity tests."""
    W, H, spp, frame = 36, 20, 3, 5
    rng = np.random.default_rng(8)
    g0, g1 = scenes.random_gbuffer(rng, W, H, rough_lo=0.05)
    g1[:, 0:2] = rng.integers(-3, 4, (W * H, 2)).astype(np.float32) + 0.25   # integer-ish motion, some off screen
    g0p = g0.copy()
    tilt = rng.random(W * H) < 0.3                                           # frame changes
    g0p[tilt, :3] = scenes.random_normals(rng, int(tilt.sum()), max_tilt=0.3)
    g0p[rng.random(W * H) < 0.1, 3] *= 2.0
    cfg = O.make_config(W, H, spp=spp, seed=31)
    cam = ocam(scenes.top_down_camera(pixel_size=0.5))
    fld = ofld(scenes.masked_lobe_field(4, n_lobes=4, kappa_hi=300.0, constant=0.02))
    gam = scenes.random_gamma(rng, W * H, k_hi=40).astype(np.float64)
    out, acc, s, img = O.frame(cfg, cam, fld, frame, g0, g1, g0p, gam)
    assert 0.05 < (acc == 0).mean() < 0.95
    idx = rng.choice(W * H, 120, replace=False)
    g, im, margin, a = O.frame_pixels(cfg, cam, fld, frame, g0, g1, g0p, gam, idx % W, idx // W, with_accept=True)
    assert np.array_equal(g, out[idx])
    assert np.array_equal(im, img[idx])
    assert np.array_equal(a, acc[idx])
    assert np.array_equal(margin, s["margin"].reshape(spp, -1)[:, idx].min(0))
