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


# ---------------------------------------------------------------------------
# State-synced parity after the first frame: before each checked frame the
# oracle gets the GPU's own Gamma(t-1), every pixel of it, so a frame starts
# from a diverse trained guide, with the screen's rejections and, in the
# orbit, the frame change of every pixel whose normal moved.
# ---------------------------------------------------------------------------
def _gamma_rows(gp, dtype):
    """The GPU's Gamma as FP64 raw-moment rows [HW, 8] (exact: the storage values)."""
    raw = host(gp.pg_get_gamma())
    if dtype == "f32":
        p = raw.view(np.float32).astype(np.float64).reshape(2, -1, 4)
        return np.concatenate([p[0], p[1]], 1)
    from test_gpu_precision import _central_to_raw_moments
    return _central_to_raw_moments(_records_to_central(raw, dtype))


def _gamma_fields(gp, dtype):
    """The GPU's Gamma in its storage form: raw moments (f32) or mean and central moments."""
    raw = host(gp.pg_get_gamma())
    if dtype == "f32":
        p = raw.view(np.float32).astype(np.float64).reshape(2, -1, 4)
        return np.concatenate([p[0], p[1]], 1)
    return _records_to_central(raw, dtype)


def _w_tolerance(cam, W, H, g0, idx):
    """Relative tolerance of the luminance mass W at each checked pixel. W is a
    plain sum of the frame's weights w = L f_r cos / p_b, so it carries their
    binary32 errors in full (the moments and pi are normalised ratios of such
    sums, where they largely cancel). Two dominate: the radiance in the far
    tail of the sharpest lobe (kappa = 500), whose exponent kappa |w - d|^2 / 2
    from a binary32 direction (|dw| <~ 2e-7) errs by up to kappa |w - d| |dw|
    <= 2e-4; and on GGX the factor G1(w_o) / cos theta_o, whose binary32
    cos theta_o (from the view ray and the normal, absolute error <~ 3e-7)
    errs relatively by 3e-7 / cos theta_o at grazing views."""
    cos_o = np.empty(len(idx))
    for k, i in enumerate(idx):
        _, d = O.camera_ray(cam, W, H, int(i % W), int(i // W))
        cos_o[k] = -(d @ g0[i, :3].astype(np.float64))
    return 2e-4 + 3e-7 / np.maximum(np.abs(cos_o), 1e-12)


def _compare_frame(dtype, got_fields, got_img, ref, rimg, margin, idx, img_rtol, w_rel):
    ok = margin >= 1e-5
    assert ok.mean() > 0.98
    if dtype == "f32":
        g = got_fields[idx][ok]
        r = ref[ok]
        rel = np.tile(np.array([1e-5] * 5 + [1e-5, 0, 0]), (len(r), 1))
        rel[:, 7] = w_rel[ok]
        tol = rel * np.abs(r) + np.array([2e-6] * 5 + [5e-6, 0, 1e-6])
        ratio = np.abs(g - r) / np.maximum(tol, 1e-300)
        assert (ratio <= 1.0).all(), ("worst ratio per field", ratio.max(0), "pixels over", (ratio > 1).sum(0))
    else:
        r16 = _round(_raw_to_central(ref), dtype)[ok]
        d = np.abs(got_fields[idx][ok] - r16)
        floor = np.zeros_like(r16)
        floor[:, 7] = 1e-6 + w_rel[ok] * np.abs(r16[:, 7])
        ratio = (d - floor) / _ulp(r16, dtype)
        assert (ratio <= 1.01).all(), ("worst ulps per field", ratio.max(0), "pixels over", (ratio > 1.01).sum(0))
        assert (got_fields[idx][ok, 6] == r16[:, 6]).all()
    assert close(got_img[idx][ok], rimg[ok], img_rtol, 1e-6) <= 1.0


def _synced(wl, dtype, checks, gbuf, grad_step=False, img_rtol=1e-4, extra_cap=None):
    """Run the workload's frames on the GPU (FP32 or FP16 Gamma; with
    grad_step one adjoint + projected Adam step after each frame, as the 4K
    leg of the benchmark), checking each frame of `checks` against the oracle
    from the GPU's Gamma(t-1) on: the screen's edges, 3000 random pixels, every
    rejected pixel and (up to extra_cap of them) pixels whose reprojected normal
    differs from their own."""
    import torch
    par, fld = wl["params"], wl["field"]
    W, H = par.width, par.height
    hw = W * H
    gp = guide(par, dtype, adam_dtype="bf16") if grad_step else guide(par, dtype)
    img = torch.empty(hw, device="cuda")
    loss, grad = torch.empty(hw, device="cuda"), torch.empty((6, hw), device="cuda")
    cfg, of = ocfg(par), ofld(fld)
    rng = np.random.default_rng(17)
    stats = []
    for t in range(max(checks) + 1):
        g0, g1, g0p = gbuf(t)
        cam = wl["camera"](t)
        if t in checks:
            prev = _gamma_rows(gp, dtype)
        gp.pg_frame(dev(g0), dev(g1), cam, dev(g0p), fld, t, img)
        if t in checks:
            gp.pg_check()
            got, gimg = _gamma_fields(gp, dtype), host(img)     # Gamma(t) as the frame left it
        if grad_step:
            gp.pg_grad(dev(g0), dev(g1), cam, fld, t, par.spp, loss=loss, grad=grad)
            gp.pg_adam_step(grad, lr=1e-2, step=t + 1)
        if t not in checks:
            continue
        _, acc, q = O.reproject(cfg, g0, g1, g0p, prev)
        moved = (acc == 1) & np.any(g0[:, :3] != g0p[np.maximum(q, 0), :3], 1)
        _, _, idx = _pixels(W, H, rng)
        rej = np.nonzero(acc == 0)[0]
        mv = np.nonzero(moved)[0]
        if extra_cap is not None and len(mv) > extra_cap:
            mv = rng.choice(mv, extra_cap, replace=False)
        idx = np.unique(np.concatenate([idx, rej, mv]))
        oc = ocam(cam)
        ref, rimg, margin = O.frame_pixels(cfg, oc, of, t, g0, g1, g0p, prev, idx % W, idx // W)
        _compare_frame(dtype, got, gimg, ref, rimg, margin, idx, img_rtol, _w_tolerance(oc, W, H, g0, idx))
        stats.append((t, len(idx), len(rej), int(moved.sum())))
    gp.close()
    return stats


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_1080p_pan_frames_1_to_3_state_synced(dtype):
    wl = scenes.workload_pan(1920, 1080, frames=4)
    stats = _synced(wl, dtype, (1, 2, 3), wl["gbuf"])
    # the pan exposes two new columns per frame: every one of them is checked
    assert all(r == 2 * 1080 for _, _, r, _ in stats)


def test_4k_orbit_frames_5_to_7_state_synced_with_gradient_steps():
    """The benchmark's 4K leg: FP16 Gamma, 4 spp, an EM frame then one adjoint
    and projected-Adam step (BF16 moments) per frame. Frames 5-7 from the
    GPU's own state, with the orbit's ~5% rejections (all checked) and its
    frame changes (20000 of them checked per frame: nearly every pixel's
    reprojected normal moves: all of the ground and the background)."""
    import torch
    wl = scenes.workload_4k()
    sc = wl["scene"]
    cache = {}

    def gbuf(t):
        if t not in cache:
            cache.clear()
            cache[t] = tuple(a.cpu().numpy() for a in sc.gbuffer_on(t, "cuda"))
        return cache[t]

    stats = _synced(wl, "f16", (5, 6, 7), gbuf, grad_step=True, img_rtol=5e-4, extra_cap=20000)
    for t, n, rej, moved in stats:
        assert 0.03 < rej / (3840 * 2160) < 0.08
        assert moved > 0.2 * 3840 * 2160
