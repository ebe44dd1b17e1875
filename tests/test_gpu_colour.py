"""Coloured radiance on the GPU (Sec. 3.1: EM samples weighted by the
radiance's luminance): the fused frame, the staged frame, the frame with
neighbour reuse and the host pipeline with a coloured field, against the
oracle and against each other. Tolerances are those of the plain frame."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2112_09728_gb300 import scenes

from _pg import close, dev, get_gamma_rows, guide, host, ocam, ocfg, ofld, set_gamma_rows

pytestmark = pytest.mark.gpu

MARGIN = 1e-5


def _scene(seed, W, H, spp=1, **kw):
    rng = np.random.default_rng(seed)
    g0, g1 = scenes.random_gbuffer(rng, W, H, glass_frac=0.1)
    gam = scenes.random_gamma(rng, W * H)
    par = dataclasses.replace(scenes.Params(W, H, spp=spp, seed=seed * 7919 + 9, transparent=1, ggx_f0=0.3), **kw)
    cam = scenes.top_down_camera(pixel_size=0.37)
    fld = scenes.coloured(scenes.masked_lobe_field(seed, n_lobes=3, kappa_hi=200.0, constant=0.05), seed)
    return rng, par, cam, fld, g0, g1, gam


def _window_any(flag, W, H, R):
    f = flag.reshape(H, W)
    out = np.zeros_like(f)
    p = np.pad(f, R)
    for dy in range(2 * R + 1):
        for dx in range(2 * R + 1):
            out |= p[dy:dy + H, dx:dx + W]
    return out.ravel()


@pytest.mark.parametrize("spp,reuse", [(1, 0), (3, 0), (1, 2)])
def test_coloured_frame_matches_oracle(spp, reuse):
    import torch
    W, H = 44, 26
    rng, par, cam, fld, g0, g1, gam = _scene(21 + spp + reuse, W, H, spp=spp, reuse_radius=reuse)
    hw = W * H
    gp = guide(par)
    set_gamma_rows(gp, gam)
    img = torch.empty(3 * hw, device="cuda")
    gp.pg_frame(dev(g0), dev(g1), cam, dev(g0), fld, 4, img)
    gp.pg_check()
    got = get_gamma_rows(gp)
    ref, _, s, rimg = O.frame(ocfg(par), ocam(cam), ofld(fld), 4, g0, g1, g0, gam.astype(np.float64))
    amb = (s["margin"] < MARGIN).reshape(spp, -1).any(0)
    ok = ~_window_any(amb, W, H, reuse) if reuse else ~amb
    assert ok.mean() > 0.9
    assert (got[ok, 6] == ref[ok, 6]).all()
    assert close(got[ok, :5], ref[ok, :5], 1e-5, 2e-6) <= 1.0
    assert close(got[ok, 5], ref[ok, 5], 1e-5, 5e-6) <= 1.0
    assert close(got[ok, 7], ref[ok, 7], 1e-4, 1e-6) <= 1.0
    gi, ri = host(img).reshape(3, hw), rimg.reshape(3, hw)
    for c in range(3):
        assert close(gi[c][~amb], ri[c][~amb], 1e-4, 1e-6) <= 1.0, c
    assert (np.abs(gi[0] - gi[2]) > 1e-3 * np.abs(gi[2])).mean() > 0.5     # the channels differ


def test_coloured_training_equals_luminance_training():
    """The guide trains on luminance alone: a coloured field and the
    monochrome field of its luminances give the same Gamma (up to the binary32
    rounding of the lobes' luminance scales)."""
    import torch
    W, H, spp = 40, 24, 2
    rng, par, cam, fld, g0, g1, gam = _scene(31, W, H, spp=spp)
    Y = np.array([0.2126, 0.7152, 0.0722])
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    lum = scenes.Field(dirs=fld.dirs, kappas=fld.kappas, amps=f32(fld.rgb) @ Y,
                       constant=float(f32(fld.constant_rgb) @ Y), mask=fld.mask)
    outs = []
    for f in (fld, lum):
        gp = guide(par)
        set_gamma_rows(gp, gam)
        gp.pg_frame(dev(g0), dev(g1), cam, dev(g0), f, 6)
        outs.append(get_gamma_rows(gp))
    assert (outs[0][:, 6] == outs[1][:, 6]).all()
    assert close(outs[0], outs[1], 1e-5, 1e-7) <= 1.0


def test_coloured_staged_and_host_paths_agree_with_fused():
    import torch
    from paper_2112_09728_gb300.guide import alloc_samples
    W, H, spp = 36, 20, 2
    rng, par, cam, fld, g0, g1, gam = _scene(41, W, H, spp=spp)
    hw = W * H
    a = guide(par)
    set_gamma_rows(a, gam)
    ia = torch.empty(3 * hw, device="cuda")
    a.pg_frame(dev(g0), dev(g1), cam, dev(g0), fld, 9, ia)
    b = guide(par)
    set_gamma_rows(b, gam)
    ib = torch.empty(3 * hw, device="cuda")
    b.pg_reproject(dev(g0), dev(g1), cam, dev(g0))
    smp = alloc_samples(spp, hw)
    b.pg_sample(dev(g0), dev(g1), cam, fld, 9, smp, ib)
    b.pg_update(dev(g0), dev(g1), cam, smp)
    assert close(host(ib), host(ia), 1e-6, 1e-9) <= 1.0
    assert close(get_gamma_rows(b), get_gamma_rows(a), 1e-5, 1e-6) <= 1.0
    c = guide(par)
    set_gamma_rows(c, gam)
    imgh = torch.zeros((1, 3 * hw))
    c.pg_frames_host(torch.from_numpy(g0).reshape(1, hw, 4).contiguous(),
                     torch.from_numpy(g1).reshape(1, hw, 4).contiguous(), [cam], fld, 9,
                     g0_prev=torch.from_numpy(g0).contiguous(), img=imgh)
    assert torch.equal(imgh[0], ia.cpu())
    assert torch.equal(c.pg_get_gamma(), a.pg_get_gamma())
