"""Parity at the benchmark's full sizes, in the configurations it times, on
a sample of pixels the oracle computes one by one (oracle.frame_pixels):

* the 1920x1080 pan workload's first frame, FP16 Gamma, one sample per pixel;
* the 3840x2160 orbit workload's first frame, FP16 Gamma, four samples.

Both start from the workload's initial guide as FP16 stores it (the oracle
gets the same rounded row, computed on the host). Pixels: the first and last
rows and columns and 3000 drawn at random. Bounds as in the precision tests:
one FP16 ulp of the oracle's result rounded once (the mass W also 1e-6
absolute), the image to 1e-4 + 1e-6; draws within 1e-5 of a decision
threshold excluded."""
import numpy as np
import pytest

import oracle as O
from paper_2112_09728_gb300 import scenes

from _pg import close, dev, guide, host, ocam, ocfg, ofld
from test_gpu_precision import _raw_to_central, _records_to_central, _round, _ulp

pytestmark = pytest.mark.gpu


def _pixels(W, H, rng, n=3000):
    i = np.concatenate([np.arange(W), (H - 1) * W + np.arange(W), np.arange(0, W * H, W),
                        np.arange(W - 1, W * H, W), rng.integers(0, W * H, n)])
    i = np.unique(i)
    return i % W, i // W, i


def _check(wl, gb, frame=0, img_rtol=1e-4):
    import torch
    par, fld, cam = wl["params"], wl["field"], wl["camera"](frame)
    W, H = par.width, par.height
    hw = W * H
    g0, g1, g0p = gb
    gp = guide(par, "f16")
    img = torch.empty(hw, device="cuda")
    gp.pg_frame(dev(g0), dev(g1), cam, dev(g0p), fld, frame, img)
    gp.pg_check()
    got = _records_to_central(host(gp.pg_get_gamma()), "f16")
    img = host(img)
    # the initial guide as FP16 stores it
    cfg = ocfg(par)
    init = O.init_gamma(cfg, 1, pi=par.init_pi)[0]
    c = _round(_raw_to_central(init[None, :])[0], "f16")
    row = np.array([c[0], c[1], c[2] + c[0] ** 2, c[3] + c[1] ** 2, c[4] + c[0] * c[1], c[5], c[6], c[7]])
    xs, ys, idx = _pixels(W, H, np.random.default_rng(W))
    ref, rimg, margin = O.frame_pixels(cfg, ocam(cam), ofld(fld), frame, g0, g1, g0p, row, xs, ys)
    ok = margin >= 1e-5
    assert ok.mean() > 0.99
    r16 = _round(_raw_to_central(ref), "f16")
    d = np.abs(got[idx] - r16)[ok]
    # the mass W (field 7) is a sum of luminance weights; where the field is
    # nearly dark its binary32 evaluation is good to ~1e-7 absolute (the
    # image's own 1e-6 floor below), which can exceed an FP16 ulp of a tiny W
    floor = np.array([0, 0, 0, 0, 0, 0, 0, 1e-6])
    assert (d <= 1.01 * _ulp(r16[ok], "f16") + floor).all(), np.max((d - floor) / _ulp(r16[ok], "f16"))
    assert (got[idx][ok, 6] == r16[ok, 6]).all()
    assert close(img[idx][ok], rimg[ok], img_rtol, 1e-6) <= 1.0


def test_1080p_pan_first_frame_fp16_sampled_pixels():
    wl = scenes.workload_pan(1920, 1080, frames=60)
    _check(wl, wl["gbuf"](0))


def test_4k_orbit_first_frame_fp16_4spp_sampled_pixels():
    # The orbit workload has GGX down to roughness 0.02 and lobes up to
    # kappa = 500. On its near-mirror pixels the estimate is the radiance along
    # the drawn direction times a smooth factor, so its relative error is
    # bounded by kappa_max |dw|; a binary32 reflection about a nearly normal
    # half vector is good to |dw| <= 1e-6: 5e-4.
    wl = scenes.workload_4k()
    _check(wl, wl["gbuf"](0), img_rtol=5e-4)
