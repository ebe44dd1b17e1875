"""Neighbour-VPL reuse (Sec. 3.2, Sec. 4.2) on the GPU: the two-pass frame
(path tracing writes one VPL per sample; training adds N picks of the
window around each pixel, weighted f / p_src) against the oracle's frame
with reuse, on random G-buffers and guide states.

Tolerances are those of the fused frame. A pixel's training reads the
samples of its whole window, so a pixel is excluded when any sample of its
(2R+1)^2 window lies within 1e-5 of a decision threshold (where the two
sides may legitimately draw differently)."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2112_09728_gb300 import _lib, scenes

from _pg import close, dev, get_gamma_rows, guide, host, ocam, ocfg, ofld, set_gamma_rows

pytestmark = pytest.mark.gpu

MARGIN = 1e-5


def _window_any(flag, W, H, R):
    f = flag.reshape(H, W)
    out = np.zeros_like(f)
    p = np.pad(f, R)
    for dy in range(2 * R + 1):
        for dx in range(2 * R + 1):
            out |= p[dy:dy + H, dx:dx + W]
    return out.ravel()


def _case(seed, W, H, spp, R, dtype="f32", k_hi=40, frame=5):
    import torch
    rng = np.random.default_rng(seed)
    g0, g1 = scenes.random_gbuffer(rng, W, H)
    gam = scenes.random_gamma(rng, W * H, k_hi=k_hi)
    par = dataclasses.replace(scenes.Params(W, H, spp=spp, seed=seed * 7919 + 11), reuse_radius=R)
    cam = scenes.top_down_camera(pixel_size=0.37)
    fld = scenes.masked_lobe_field(seed, n_lobes=3, kappa_hi=200.0, constant=0.05)
    gp = guide(par, dtype)
    set_gamma_rows(gp, gam)
    img = torch.empty(W * H, device="cuda")
    gp.pg_frame(dev(g0), dev(g1), cam, dev(g0), fld, frame, img)
    gp.pg_check()
    got = get_gamma_rows(gp)
    ref, acc, s, rimg = O.frame(ocfg(par), ocam(cam), ofld(fld), frame, g0, g1, g0, gam.astype(np.float64))
    amb = (s["margin"] < MARGIN).reshape(spp, -1).any(0)
    return got, host(img), ref, rimg, amb, gam


# the window tile fits shared memory for all but (4, 2), which reads the
# neighbours' samples from the global buffers: both training-pass variants
@pytest.mark.parametrize("spp,R", [(1, 2), (2, 1), (1, 3), (3, 1), (4, 2)])
def test_reuse_frame_matches_oracle(spp, R):
    W, H = 48, 30
    got, img, ref, rimg, amb, gam = _case(21 + R, W, H, spp, R)
    ok = ~_window_any(amb, W, H, R)
    assert ok.mean() > 0.8
    assert (got[ok, 6] == ref[ok, 6]).all()
    assert close(got[ok, :5], ref[ok, :5], 1e-5, 2e-6) <= 1.0
    assert close(got[ok, 5], ref[ok, 5], 1e-5, 5e-6) <= 1.0
    assert close(got[ok, 7], ref[ok, 7], 1e-4, 1e-6) <= 1.0
    assert close(img[~amb], rimg[~amb], 1e-4, 1e-6) <= 1.0


def test_reuse_changes_the_update():
    # the same case without reuse: the trained masses differ for most pixels
    W, H = 48, 30
    got, _, _, _, amb, gam = _case(23, W, H, 1, 2)
    rng = np.random.default_rng(23)
    par = scenes.Params(W, H, seed=23 * 7919 + 11)
    g0, g1 = scenes.random_gbuffer(rng, W, H)
    gam0 = scenes.random_gamma(rng, W * H, k_hi=40)
    ref0, _, _, _ = O.frame(ocfg(par), ocam(scenes.top_down_camera(pixel_size=0.37)),
                            ofld(scenes.masked_lobe_field(23, n_lobes=3, kappa_hi=200.0, constant=0.05)),
                            5, g0, g1, g0, gam0.astype(np.float64))
    assert (np.abs(got[:, 7] - ref0[:, 7]) > 1e-3 * np.abs(ref0[:, 7])).mean() > 0.5


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_reuse_frame_reduced_precision_to_one_ulp(dtype):
    """From a Gamma exactly representable in the storage type, the GPU's
    frame with reuse and the oracle's, rounded once to that type, agree to one
    unit in its last place (the binary32 result may sit within ~1e-6 of a
    rounding boundary)."""
    import torch
    from test_gpu_precision import _central_to_raw_moments, _raw_to_central, _record_bytes, \
        _records_to_central, _round, _ulp
    W, H, R = 40, 24, 2
    hw = W * H
    rng = np.random.default_rng(41)
    g0, g1 = scenes.random_gbuffer(rng, W, H, rough_lo=0.05)
    mx, my = rng.uniform(0.05, 0.95, (2, hw))
    sx, sy = np.exp(rng.uniform(np.log(0.03), np.log(0.4), (2, hw)))
    rho = rng.uniform(-0.8, 0.8, hw)
    cen = np.stack([mx, my, sx * sx, sy * sy, rho * sx * sy, rng.uniform(0.05, 0.95, hw),
                    rng.integers(0, 33, hw).astype(float), rng.uniform(0.1, 3.0, hw)], 1)
    cen = _round(cen, dtype)
    par = dataclasses.replace(scenes.Params(W, H, seed=4243), reuse_radius=R)
    cam = scenes.top_down_camera(pixel_size=0.5)
    fld = scenes.masked_lobe_field(9, n_lobes=3, kappa_hi=150.0, constant=0.05)
    gp = guide(par, dtype)
    gp.pg_set_gamma(torch.from_numpy(_record_bytes(cen, dtype)).cuda())
    img = torch.empty(hw, device="cuda")
    gp.pg_frame(dev(g0), dev(g1), cam, dev(g0), fld, 2, img)
    gp.pg_check()
    got = _records_to_central(host(gp.pg_get_gamma()), dtype)
    ref_raw, _, s, rimg = O.frame(ocfg(par), ocam(cam), ofld(fld), 2, g0, g1, g0, _central_to_raw_moments(cen))
    ref = _round(_raw_to_central(ref_raw), dtype)
    ok = ~_window_any((s["margin"] < MARGIN).reshape(1, -1).any(0), W, H, R)
    assert ok.mean() > 0.9
    d = np.abs(got - ref)[ok]
    assert (d <= 1.01 * _ulp(ref[ok], dtype)).all(), np.max(d / _ulp(ref[ok], dtype))
    assert (got[ok, 6] == ref[ok, 6]).all()


def test_staged_calls_and_noalloc_refuse_reuse():
    import torch
    from paper_2112_09728_gb300.guide import alloc_samples, make_config, pg_frame_noalloc
    W, H = 16, 8
    rng = np.random.default_rng(3)
    g0, g1 = scenes.random_gbuffer(rng, W, H)
    par = dataclasses.replace(scenes.Params(W, H), reuse_radius=1)
    gp = guide(par)
    cam, fld = scenes.top_down_camera(), scenes.two_lobe_field(3)
    with pytest.raises(_lib.PgError) as e:
        gp.pg_reproject(dev(g0), dev(g1), cam, dev(g0))
    assert e.value.status == _lib.PG_ERR_ARG
    gp.pg_frame(dev(g0), dev(g1), cam, dev(g0), fld, 0)     # the context stays usable
    gp.pg_check()
    cfg = make_config(W, H, reuse_radius=1)
    gin = torch.zeros(W * H * 32, dtype=torch.uint8, device="cuda")
    gout = torch.zeros_like(gin)
    with pytest.raises((_lib.PgError, ValueError)):
        pg_frame_noalloc(cfg, dev(g0), dev(g1), cam, dev(g0), fld, 0, gin, gout, alloc_samples(1, W * H))
