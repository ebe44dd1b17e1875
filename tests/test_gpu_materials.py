"""Transparent surfaces (Sec. 5: guiding off) and the GGX Fresnel term on the
GPU, against the oracle, on random G-buffers with a quarter of the pixels
transparent and Schlick's F0 = 0.04 on the GGX pixels.

Tolerances are those of the plain pass (test_gpu_parity.py): evaluation at
the same input 1e-5 relative plus the value's gradient times the direction
error; fused frame 1e-5 + 2e-6 on moments; draws within 1e-5 of a decision
threshold (for a transparent pixel: the Fresnel reflectance against its
uniform) excluded."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2112_09728_gb300 import scenes

from _pg import close, dev, get_gamma_rows, guide, host, ocam, ocfg, ofld, set_gamma_rows
from test_gpu_parity import oracle_grad_norm

pytestmark = pytest.mark.gpu

MARGIN = 1e-5


def _scene(seed, W, H, spp=1, glass=0.25, f0=0.04):
    rng = np.random.default_rng(seed)
    g0, g1 = scenes.random_gbuffer(rng, W, H, ggx_frac=0.5, rough_lo=0.05, glass_frac=glass)
    gam = scenes.random_gamma(rng, W * H)
    par = dataclasses.replace(scenes.Params(W, H, spp=spp, seed=seed * 7919 + 5), ggx_f0=f0, transparent=1)
    cam = scenes.top_down_camera(pixel_size=0.37)
    fld = scenes.masked_lobe_field(seed, n_lobes=3, kappa_hi=200.0, constant=0.05)
    return rng, par, cam, fld, g0, g1, gam


def test_frame_with_transparent_pixels_and_fresnel_matches_oracle():
    import torch
    W, H, spp = 45, 31, 2
    rng, par, cam, fld, g0, g1, gam = _scene(11, W, H, spp=spp)
    glass = g1[:, 2] <= -1.5
    assert 0.15 < glass.mean() < 0.35
    gp = guide(par)
    set_gamma_rows(gp, gam)
    img = torch.empty(W * H, device="cuda")
    gp.pg_frame(dev(g0), dev(g1), cam, dev(g0), fld, 3, img)
    gp.pg_check()
    got = get_gamma_rows(gp)
    ref, _, s, rimg = O.frame(ocfg(par), ocam(cam), ofld(fld), 3, g0, g1, g0, gam.astype(np.float64))
    ok = ~(s["margin"] < MARGIN).reshape(spp, -1).any(0)
    assert ok.mean() > 0.99
    assert (got[ok, 6] == ref[ok, 6]).all()
    assert close(got[ok, :5], ref[ok, :5], 1e-5, 2e-6) <= 1.0
    assert close(got[ok, 5], ref[ok, 5], 1e-5, 5e-6) <= 1.0
    assert close(got[ok, 7], ref[ok, 7], 1e-4, 1e-6) <= 1.0
    assert close(host(img)[ok], rimg[ok], 1e-4, 1e-6) <= 1.0
    # transparent pixels keep their guide (stored exactly as set)
    g32 = gam.astype(np.float64)
    assert np.array_equal(got[glass], g32[glass])


def test_transparent_sample_records_match_oracle():
    import torch
    from paper_2112_09728_gb300.guide import alloc_samples
    W, H, spp = 33, 17, 4
    rng, par, cam, fld, g0, g1, gam = _scene(12, W, H, spp=spp)
    hw = W * H
    gp = guide(par)
    set_gamma_rows(gp, gam)
    gp.pg_reproject(dev(g0), dev(g1), cam, dev(g0))
    smp = alloc_samples(spp, hw)
    gp.pg_sample(dev(g0), dev(g1), cam, fld, 5, smp)
    got = {k: host(v) for k, v in smp.items()}
    cfg, oc, of = ocfg(par), ocam(cam), ofld(fld)
    ref, _ = O.sample(cfg, oc, of, 5, g0, g1, gam.astype(np.float64))
    glass = np.tile(g1[:, 2] <= -1.5, spp)
    ok = ~(ref["margin"] < MARGIN)
    assert (got["strategy"][ok] == ref["strategy"][ok]).all()
    sel = glass & ok
    assert sel.sum() > 100
    assert (got["strategy"][sel] == 3).all()
    assert (got["mis"][sel] == 1.0).all() and (got["pdf"][sel] == 0.0).all()
    wg = np.stack([got["wx"], got["wy"], got["wz"]], -1).astype(np.float64)
    wr = np.stack([ref["wx"], ref["wy"], ref["wz"]], -1)
    dw = np.linalg.norm(wg - wr, axis=-1)
    assert dw[sel].max() < 2e-6
    assert (wr[sel, 2] < 0).any() and (wr[sel, 2] > 0).any()      # both refractions and reflections
    grad = oracle_grad_norm(cfg, oc, of, g0, g1, gam.astype(np.float64), wr.reshape(spp, hw, 3))
    gL = grad["radiance"].reshape(-1)
    a = np.tile(g1[:, 3].astype(np.float64), spp)
    assert close(got["estimate"][sel], ref["estimate"][sel], 1e-5, (2 * a * gL * np.maximum(dw, 4e-7))[sel]) <= 1.0


def test_eval_and_adjoint_give_transparent_pixels_nothing():
    W, H, n = 37, 23, 6
    rng, par, cam, fld, g0, g1, gam = _scene(13, W, H)
    glass = g1[:, 2] <= -1.5
    dirs = scenes.random_directions(rng, n, W * H)
    gp = guide(par)
    set_gamma_rows(gp, gam)
    out = {k: host(v).astype(np.float64) for k, v in gp.pg_eval(dev(g0), dev(g1), cam, fld, dev(dirs)).items()}
    cfg, oc, of = ocfg(par), ocam(cam), ofld(fld)
    ref = O.evaluate(cfg, oc, of, g0, g1, gam.astype(np.float64), dirs)
    grad = oracle_grad_norm(cfg, oc, of, g0, g1, gam.astype(np.float64), dirs)
    for k in ref:
        scale = np.abs(ref["pmix"]) if k in ("pg", "pb", "pmix") else (1.0 if k.startswith("w_") else 0.0)
        # a transparent pixel's guide density enters nothing (p_mix = 0 there):
        # compared on the other pixels only, where p_mix scales its tolerance
        cols = ~glass if k == "pg" else np.ones_like(glass)
        assert close(out[k][:, cols], ref[k][:, cols], 1e-5,
                     (1e-6 * scale + 4e-7 * grad[k] + 1e-30)[:, cols]) <= 1.0, k
    for k in ("pb", "pmix", "fcos"):
        assert (out[k][:, glass] == 0).all()
    loss, g = gp.pg_grad(dev(g0), dev(g1), cam, fld, 7, 16)
    loss, g = host(loss), host(g)
    assert (loss[glass] == 0).all() and (g[:, glass] == 0).all()
    assert (loss[~glass] > 0).mean() > 0.9


def test_transparent_code_is_lambertian_unless_enabled():
    """With the transparent material off (the default), the fused kernel is
    the one without its code and a roughness code of -2 renders exactly as -1."""
    import torch
    W, H, spp = 40, 24, 1
    rng, par, cam, fld, g0, g1, gam = _scene(14, W, H, spp=spp)
    par = dataclasses.replace(par, transparent=0)
    g1l = g1.copy()
    g1l[g1l[:, 2] <= -1.5, 2] = -1.0
    outs = []
    for gb in (g1, g1l):
        gp = guide(par)
        set_gamma_rows(gp, gam)
        img = torch.empty(W * H, device="cuda")
        gp.pg_frame(dev(g0), dev(gb), cam, dev(g0), fld, 3, img)
        outs.append((gp.pg_get_gamma().clone(), img.clone()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
