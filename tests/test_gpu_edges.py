"""Edge cases and degenerate inputs of the guide pass on the GPU, against the
oracle: the smallest screens (1x1, one row, one column), a field of zero
radiance (no sample carries luminance, so nothing trains), every pixel
rejected by the reprojection (all guides re-initialised, guiding off), views
from below the surface (every draw wasted), many samples per pixel, and the
largest screen the tests allocate (4096 x 4096), checked pixel by pixel on a
sample of pixels. Tolerances are those of the plain frame."""
import numpy as np
import pytest

import oracle as O
from paper_2112_09728_gb300 import scenes

from _pg import close, dev, get_gamma_rows, guide, host, ocam, ocfg, ofld, set_gamma_rows

pytestmark = pytest.mark.gpu

MARGIN = 1e-5


def _frame_both(par, cam, fld, g0, g1, g0p, gam, frame=3, dtype="f32"):
    import torch
    hw = par.width * par.height
    gp = guide(par, dtype)
    set_gamma_rows(gp, gam)
    img = torch.empty(hw, device="cuda")
    gp.pg_frame(dev(g0), dev(g1), cam, dev(g0p), fld, frame, img)
    gp.pg_check()
    got = get_gamma_rows(gp)
    ref, acc, s, rimg = O.frame(ocfg(par), ocam(cam), ofld(fld), frame, g0, g1, g0p, gam.astype(np.float64))
    ok = ~(s["margin"] < MARGIN).reshape(par.spp, -1).any(0)
    return got, host(img), ref, rimg, acc, s, ok


def _check(got, img, ref, rimg, ok):
    assert (got[ok, 6] == ref[ok, 6]).all()
    assert close(got[ok, :5], ref[ok, :5], 1e-5, 2e-6) <= 1.0
    assert close(got[ok, 5], ref[ok, 5], 1e-5, 5e-6) <= 1.0
    assert close(got[ok, 7], ref[ok, 7], 1e-4, 1e-6) <= 1.0
    assert close(img[ok], rimg[ok], 1e-4, 1e-6) <= 1.0


@pytest.mark.parametrize("W,H,spp", [(1, 1, 1), (1, 1, 5), (257, 1, 2), (1, 300, 1)])
def test_smallest_screens(W, H, spp):
    rng = np.random.default_rng(W * 1000 + H)
    g0, g1 = scenes.random_gbuffer(rng, W, H)
    gam = scenes.random_gamma(rng, W * H)
    par = scenes.Params(W, H, spp=spp, seed=5)
    cam = scenes.top_down_camera(pixel_size=0.5)
    fld = scenes.masked_lobe_field(3, n_lobes=3, constant=0.05)
    got, img, ref, rimg, _, _, ok = _frame_both(par, cam, fld, g0, g1, g0, gam)
    _check(got, img, ref, rimg, ok)


def test_zero_radiance_trains_nothing():
    W, H = 40, 20
    rng = np.random.default_rng(1)
    g0, g1 = scenes.random_gbuffer(rng, W, H)
    gam = scenes.random_gamma(rng, W * H)
    gam[:, 6] = np.abs(gam[:, 6])
    par = scenes.Params(W, H, spp=3, seed=6)
    fld = scenes.Field(dirs=np.zeros((0, 3)), kappas=np.zeros(0), amps=np.zeros(0), constant=0.0)
    got, img, ref, rimg, _, _, ok = _frame_both(par, scenes.top_down_camera(), fld, g0, g1, g0, gam)
    assert (img == 0).all() and (rimg == 0).all()
    # b = 0 everywhere: the stored guide is the reprojected one, k included
    assert np.array_equal(got, gam.astype(np.float64))
    _check(got, img, ref, rimg, ok)


def test_every_pixel_rejected():
    W, H = 33, 17
    rng = np.random.default_rng(2)
    g0, g1 = scenes.random_gbuffer(rng, W, H)
    g0p = g0.copy()
    g0p[:, 3] *= 3.0                 # depth test fails everywhere
    gam = scenes.random_gamma(rng, W * H)
    par = scenes.Params(W, H, spp=2, seed=7)
    got, img, ref, rimg, acc, s, ok = _frame_both(par, scenes.top_down_camera(), scenes.two_lobe_field(2),
                                                  g0, g1, g0p, gam)
    assert (acc == 0).all()
    st = s["strategy"] & 3
    assert not (st == 1).any()       # guiding off on fresh history
    assert (got[:, 6] <= 1).all()
    _check(got, img, ref, rimg, ok)


def test_views_from_below_waste_every_draw():
    W, H = 24, 12
    rng = np.random.default_rng(3)
    g0, g1 = scenes.random_gbuffer(rng, W, H, ggx_frac=0.5)
    g0[:, :3] *= -1.0                # normals facing away from the camera
    gam = scenes.random_gamma(rng, W * H)
    par = scenes.Params(W, H, spp=2, seed=8)
    got, img, ref, rimg, _, s, ok = _frame_both(par, scenes.top_down_camera(), scenes.two_lobe_field(2),
                                                g0, g1, g0, gam)
    assert (img == 0).all() and (rimg == 0).all()
    _check(got, img, ref, rimg, ok)


def test_many_samples_per_pixel():
    W, H, spp = 12, 10, 256
    rng = np.random.default_rng(4)
    g0, g1 = scenes.random_gbuffer(rng, W, H)
    gam = scenes.random_gamma(rng, W * H)
    par = scenes.Params(W, H, spp=spp, seed=9)
    got, img, ref, rimg, _, _, ok = _frame_both(par, scenes.top_down_camera(pixel_size=0.4),
                                                scenes.masked_lobe_field(5, n_lobes=4), g0, g1, g0, gam)
    assert ok.mean() > 0.5
    # 256 binary32 Kahan-compensated sums: the same bounds
    _check(got, img, ref, rimg, ok)
