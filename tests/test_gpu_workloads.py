"""The 4K workload's per-frame step at reduced size: a pinhole camera orbiting
over a normal-mapped ground with 16 occluding quads (about 5% of pixels fail
the reprojection test each frame), GGX everywhere, 8 lobes, 4 spp; each frame
runs the EM pass and then one gradient step (the second-moment adjoint and a
projected Adam step).

* One frame from a seeded Gamma: GPU (pg_frame, pg_grad, pg_adam_step) against
  the oracle's composition (frame, second_moment, adam). Adam's first step is
  lr * g / (|g| + eps), so a gradient component near zero has an ill-posed
  sign: the adjoint agrees with the oracle to ~1e-3 of a pixel's largest
  component, so pixels with a nonzero component below 1e-4 of their largest
  are excluded, as are pixels with a draw within 1e-5 of a decision threshold.
* Eight FP16 frames on the GPU: finite, in bounds, the expected rejection rate.
"""
import numpy as np
import pytest

import oracle as O
from paper_2112_09728_gb300 import scenes

from _pg import close, dev, get_gamma_rows, guide, host, ocam, ocfg, ofld, set_gamma_rows

pytestmark = pytest.mark.gpu


def test_quad_workload_frame_plus_gradient_step_matches_oracle():
    import torch
    W, H, spp, t = 96, 54, 4, 7
    wl = scenes.workload_4k(W, H, spp=spp, frames=16)
    par, fld = wl["params"], wl["field"]
    hw = W * H
    rng = np.random.default_rng(71)
    gam = scenes.random_gamma(rng, hw, k_hi=32)
    g0, g1, g0p = wl["gbuf"](t)
    cam = wl["camera"](t)
    gp = guide(par)
    set_gamma_rows(gp, gam)
    img = torch.empty(hw, device="cuda")
    gp.pg_frame(dev(g0), dev(g1), cam, dev(g0p), fld, t, img)
    _, grad = gp.pg_grad(dev(g0), dev(g1), cam, fld, t, spp)
    gp.pg_adam_step(grad, lr=1e-2, step=1)
    gp.pg_check()
    got = get_gamma_rows(gp)

    cfg, oc, of = ocfg(par), ocam(cam), ofld(fld)
    ref, acc, s, rimg = O.frame(cfg, oc, of, t, g0, g1, g0p, gam.astype(np.float64))
    th = O.theta_from_gamma(cfg, ref)
    _, rgrad, margin = O.second_moment(cfg, oc, of, t, spp, g0, g1, th)
    ref, _, _ = O.adam(cfg, ref, rgrad, np.zeros((hw, 6)), np.zeros((hw, 6)), 1e-2, 0.9, 0.999, 1e-8, 1)

    assert 0.01 < 1 - acc.mean() < 0.12
    amb = (s["margin"] < 1e-5).reshape(spp, -1).any(0) | (margin < 1e-5)
    gmax = np.abs(rgrad).max(1, keepdims=True)
    small = ((np.abs(rgrad) < 1e-4 * gmax) & (np.abs(rgrad) > 0)).any(1)
    ok = ~amb & ~small
    assert ok.mean() > 0.5
    assert (got[ok, 6] == ref[ok, 6]).all()
    assert close(got[ok, :6], ref[ok, :6], 1e-4, 2e-6) <= 1.0
    assert close(host(img)[ok], rimg[ok], 1e-4, 1e-6) <= 1.0


def test_quad_workload_eight_fp16_frames_with_gradient_steps():
    import torch
    W, H, spp = 192, 108, 4
    wl = scenes.workload_4k(W, H, spp=spp, frames=16)
    par, fld, sc = wl["params"], wl["field"], wl["scene"]
    hw = W * H
    gp = guide(par, "f16")
    img = torch.empty(hw, device="cuda")
    acc = torch.empty(hw, dtype=torch.uint8, device="cuda")
    rates = []
    from paper_2112_09728_gb300.guide import alloc_samples
    s = alloc_samples(spp, hw)
    for t in range(8):
        g0, g1, g0p = sc.gbuffer_on(t, "cuda")
        cam = wl["camera"](t)
        # the staged path exposes the accept mask; the fused frame is the same pass
        gp.pg_reproject(g0, g1, cam, g0p, acc)
        gp.pg_sample(g0, g1, cam, fld, t, s, img)
        gp.pg_update(g0, g1, cam, s)
        rates.append(1.0 - host(acc).mean())
        _, grad = gp.pg_grad(g0, g1, cam, fld, t, spp)
        gp.pg_adam_step(grad, lr=1e-2, step=t + 1)
    gp.pg_check()
    rows = get_gamma_rows(gp)
    assert np.isfinite(rows).all()
    assert (rows[:, 5] >= 0.05 - 1e-3).all() and (rows[:, 5] <= 0.95 + 1e-3).all()
    assert (rows[:, :2] >= 0).all() and (rows[:, :2] <= 1).all()
    assert 0.02 < np.mean(rates[1:]) < 0.1
    assert np.isfinite(host(img)).all()
