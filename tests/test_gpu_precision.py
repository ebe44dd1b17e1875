"""The reduced-precision form of the pass: Gamma stored in FP16 or BF16 as
{mu_x, mu_y, s_xx, s_yy, s_xy, pi, k, W} (mean and central second moments),
all arithmetic in binary32 with Kahan-compensated E-step sums.

* One frame from a Gamma that is exactly representable in the storage type:
  the GPU computes in binary32 and rounds once; the oracle computes in binary64
  and the test rounds once to the same type. The two may differ where the
  binary32 result lies within ~1e-6 of a rounding boundary, so the bound is one
  unit in the last place of the storage type.
* The 64x64, 8-frame workload in FP32, FP16 and BF16 against the FP64 oracle:
  per-parameter error and image MSE are reported and bounded.
"""
import numpy as np
import pytest

import oracle as O
from paper_2112_09728_gb300 import scenes

from _pg import close, dev, get_gamma_rows, guide, host, ocam, ocfg, ofld, set_gamma_rows

pytestmark = pytest.mark.gpu


def _round(x, dtype):
    """Round to nearest in the storage type; FP16 saturates at +-65504 as the store does."""
    import torch
    t = torch.from_numpy(np.asarray(x, np.float64))
    if dtype == "f16":
        return t.clamp(-65504.0, 65504.0).to(torch.float16).to(torch.float64).numpy()
    return t.to(torch.bfloat16).to(torch.float64).numpy()


def _ulp(x, dtype):
    """Unit in the last place of the storage type at |x| (subnormal floor)."""
    mant = 10 if dtype == "f16" else 7
    tiny = 2.0 ** -24 if dtype == "f16" else 2.0 ** -133
    e = np.floor(np.log2(np.maximum(np.abs(x), 1e-300)))
    return np.maximum(2.0 ** (e - mant), tiny)


def _record_bytes(central, dtype):
    """[HW, 8] central-form rows -> raw 16-byte records (uint8 [HW*16])."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(central, np.float64))
    h = t.to(torch.float16) if dtype == "f16" else t.to(torch.bfloat16)
    return h.contiguous().view(torch.uint8).reshape(-1).numpy()


def _records_to_central(raw, dtype):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(raw)).view(torch.float16 if dtype == "f16" else torch.bfloat16)
    return t.to(torch.float64).numpy().reshape(-1, 8)


def _central_to_raw_moments(c):
    mx, my, sxx, syy, sxy = c[:, 0], c[:, 1], c[:, 2], c[:, 3], c[:, 4]
    return np.stack([mx, my, sxx + mx * mx, syy + my * my, sxy + mx * my, c[:, 5], c[:, 6], c[:, 7]], 1)


def _raw_to_central(r):
    mx, my = r[:, 0], r[:, 1]
    return np.stack([mx, my, r[:, 2] - mx * mx, r[:, 3] - my * my, r[:, 4] - mx * my, r[:, 5], r[:, 6], r[:, 7]], 1)


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_reduced_precision_frame_matches_oracle_to_one_ulp(dtype):
    import torch
    W, H, spp = 40, 27, 2
    rng = np.random.default_rng(31)
    g0, g1 = scenes.random_gbuffer(rng, W, H, rough_lo=0.05)
    hw = W * H
    mx, my = rng.uniform(0.05, 0.95, (2, hw))
    sx, sy = np.exp(rng.uniform(np.log(0.03), np.log(0.4), (2, hw)))
    rho = rng.uniform(-0.8, 0.8, hw)
    cen = np.stack([mx, my, sx * sx, sy * sy, rho * sx * sy, rng.uniform(0.05, 0.95, hw),
                    rng.integers(0, 33, hw).astype(float), rng.uniform(0.1, 3.0, hw)], 1)
    cen = _round(cen, dtype)                     # exactly representable in storage
    par = scenes.Params(W, H, spp=spp, seed=4242)
    cam = scenes.top_down_camera(pixel_size=0.5)
    fld = scenes.masked_lobe_field(9, n_lobes=3, kappa_hi=150.0, constant=0.05)
    gp = guide(par, dtype)
    gp.pg_set_gamma(torch.from_numpy(_record_bytes(cen, dtype)).cuda())
    img = torch.empty(hw, device="cuda")
    gp.pg_frame(dev(g0), dev(g1), cam, dev(g0), fld, 1, img)
    gp.pg_check()
    got = _records_to_central(host(gp.pg_get_gamma()), dtype)
    ref_raw, _, s, rimg = O.frame(ocfg(par), ocam(cam), ofld(fld), 1, g0, g1, g0, _central_to_raw_moments(cen))
    ref = _round(_raw_to_central(ref_raw), dtype)
    ok = ~(s["margin"] < 1e-5).reshape(spp, -1).any(0)
    assert ok.mean() > 0.99
    d = np.abs(got - ref)[ok]
    assert (d <= 1.01 * _ulp(ref[ok], dtype)).all(), np.max(d / _ulp(ref[ok], dtype))
    assert (got[ok, 6] == ref[ok, 6]).all()
    assert close(host(img)[ok], rimg[ok], 1e-4, 1e-6) <= 1.0


def test_precision_report_small_workload():
    """64x64, 1 spp, 8 frames: each storage form against the FP64 oracle run
    forward on its own, and FP16/BF16 against the FP32 pass."""
    import torch
    wl = scenes.workload_small()
    par, cam, fld = wl["params"], wl["camera"], wl["field"]
    g0, g1, g0p = wl["gbuf"](0)
    cfg = ocfg(par)
    ref = O.init_gamma(cfg, par.width * par.height, pi=par.init_pi)
    imgs_ref = []
    amb = np.zeros(par.width * par.height, bool)
    for t in range(wl["frames"]):
        ref, _, s, rimg = O.frame(cfg, ocam(cam), ofld(fld), t, g0, g1, g0p, ref)
        amb |= (s["margin"] < 1e-5).reshape(par.spp, -1).any(0)
        imgs_ref.append(rimg)
    ok = ~amb                 # pixels whose decisions never came within 1e-5 of a threshold
    out = {}
    for dtype in ("f32", "f16", "bf16"):
        gp = guide(par, dtype)
        img = torch.empty(par.width * par.height, device="cuda")
        imgs = []
        for t in range(wl["frames"]):
            gp.pg_frame(dev(g0), dev(g1), cam, dev(g0p), fld, t, img)
            imgs.append(host(img).astype(np.float64))
        gp.pg_check()
        out[dtype] = (_raw_to_central(get_gamma_rows(gp)), np.array(imgs))
    rc = _raw_to_central(ref)
    names = ("mu_x", "mu_y", "s_xx", "s_yy", "s_xy", "pi", "k", "W")
    report = {}
    for dtype, (c, im) in out.items():
        d = np.abs(c - rc)[ok]
        err, err99 = d.max(0), np.percentile(d, 99, axis=0)
        mse = float(((im - np.array(imgs_ref))[:, ok] ** 2).mean())
        report[dtype] = (err, err99, mse)
        print(dtype, "vs FP64 oracle: max |err|", dict(zip(names, np.round(err, 7))), "99th pct",
              dict(zip(names, np.round(err99, 7))), "image MSE:", mse)
    for dtype in ("f16", "bf16"):
        e = np.abs(out[dtype][0] - out["f32"][0])[ok].max(0)
        print(dtype, "max |err| vs FP32 pass:", dict(zip(names, np.round(e, 7))))
    # FP32 tracks the oracle closely. In FP16/BF16 the stored pi differs from
    # the FP64 one by a storage ulp, so a few strategy choices flip and those
    # pixels take other samples: their bound is on the 99th percentile.
    assert report["f32"][0][:6].max() < 2e-4
    assert report["f16"][1][:6].max() < 5e-3
    assert report["bf16"][1][:6].max() < 5e-2


# ---------------------------------------------------------------------------
# Stochastic rounding of the 16-bit store
# ---------------------------------------------------------------------------
def _neighbours(v, dtype):
    """The storage-type neighbours of float64 values v: lo toward zero, hi away."""
    import torch
    tt = torch.float16 if dtype == "f16" else torch.bfloat16
    x = torch.from_numpy(np.asarray(v, np.float64))
    h = x.to(tt)
    bits = h.view(torch.int16).to(torch.int32) & 0xFFFF
    mag = bits & 0x7FFF
    sign = bits & 0x8000
    over = h.to(torch.float64).abs() > x.abs()
    lo_mag = torch.where(over, mag - 1, mag)
    hi_mag = lo_mag + 1

    def val(m):
        b = (sign | m).to(torch.int32)
        b = torch.where(b >= 0x8000, b - 0x10000, b).to(torch.int16)
        return b.view(tt).to(torch.float64).numpy()
    lo, hi = val(lo_mag), val(hi_mag)
    lo = np.where(np.asarray(v) == 0, 0.0, lo)
    return lo, hi


def _sr_reference(v, r16, dtype):
    """Stochastic rounding from its definition: hi with probability
    f = (|v| - |lo|) / (|hi| - |lo|), taken as U >= 1 - f for the uniform U
    the random bits give (13 of them for FP16, all 16 for BF16)."""
    v = np.asarray(v, np.float64)
    lo, hi = _neighbours(v, dtype)
    span = np.abs(hi) - np.abs(lo)
    f = np.where(span > 0, (np.abs(v) - np.abs(lo)) / np.where(span > 0, span, 1.0), 0.0)
    u = (r16 >> 3) / 8192.0 if dtype == "f16" else r16 / 65536.0
    return np.where(u >= 1.0 - f, hi, lo)


def _sr_bits(cfg, frame, hw):
    ctr = np.zeros((hw, 4), np.uint32)
    ctr[:, 0] = np.arange(hw)
    ctr[:, 1] = frame
    ctr[:, 3] = 5
    w = O.philox(ctr, (cfg.seed_lo, cfg.seed_hi)).astype(np.int64)
    # field j: bits 16 (j mod 2) and up of word j / 2
    return np.stack([(w[:, j // 2] >> (16 * (j % 2))) & 0xFFFF for j in range(8)], 1)


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_stochastic_rounding_frame_matches_reference_to_one_ulp(dtype):
    import dataclasses
    import torch
    W, H, spp, frame = 40, 27, 2, 3
    rng = np.random.default_rng(32)
    g0, g1 = scenes.random_gbuffer(rng, W, H, rough_lo=0.05)
    hw = W * H
    mx, my = rng.uniform(0.05, 0.95, (2, hw))
    sx, sy = np.exp(rng.uniform(np.log(0.03), np.log(0.4), (2, hw)))
    rho = rng.uniform(-0.8, 0.8, hw)
    cen = np.stack([mx, my, sx * sx, sy * sy, rho * sx * sy, rng.uniform(0.05, 0.95, hw),
                    rng.integers(0, 33, hw).astype(float), rng.uniform(0.1, 3.0, hw)], 1)
    cen = _round(cen, dtype)
    par = scenes.Params(W, H, spp=spp, seed=4244)
    cam = scenes.top_down_camera(pixel_size=0.5)
    fld = scenes.masked_lobe_field(9, n_lobes=3, kappa_hi=150.0, constant=0.05)
    from paper_2112_09728_gb300.guide import GuidePass
    gp = GuidePass(W, H, spp=spp, gamma_dtype=dtype, seed=par.seed, init_pi=par.init_pi, stochastic_round=1)
    gp.pg_set_gamma(torch.from_numpy(_record_bytes(cen, dtype)).cuda())
    gp.pg_frame(dev(g0), dev(g1), cam, dev(g0), fld, frame)
    gp.pg_check()
    got = _records_to_central(host(gp.pg_get_gamma()), dtype)
    cfg = ocfg(par)
    ref_raw, _, s, _ = O.frame(cfg, ocam(cam), ofld(fld), frame, g0, g1, g0, _central_to_raw_moments(cen))
    ref64 = _raw_to_central(ref_raw)
    ref = _sr_reference(ref64, _sr_bits(cfg, frame, hw), dtype)
    ok = ~(s["margin"] < 1e-5).reshape(spp, -1).any(0)
    d = np.abs(got - ref)[ok]
    assert (d <= 1.01 * _ulp(ref[ok], dtype)).all(), np.max(d / _ulp(ref[ok], dtype))
    assert (got[ok, 6] == ref[ok, 6]).all()
    # the rounding is live: of the fields the update moved, about a quarter
    # round differently from round-to-nearest (probability min(f, 1 - f))
    rn = _round(ref64, dtype)
    moved = (np.abs(ref64 - cen) > 0)[ok]
    moved[:, 6] = False
    assert moved.mean() > 0.2
    assert (got[ok] != rn[ok])[moved].mean() > 0.15


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_stochastic_rounding_is_unbiased_on_the_gpu(dtype):
    """The same EM update from the same state and samples, rounded with 256
    different sets of random bits: the mean of the stored values approaches
    the binary32 update, well inside the half-ulp bias of rounding to
    nearest."""
    import torch
    from paper_2112_09728_gb300.guide import GuidePass
    W, H, spp, n = 24, 16, 2, 256
    hw = W * H
    rng = np.random.default_rng(33)
    g0, g1 = scenes.random_gbuffer(rng, W, H, rough_lo=0.05)
    cen = _round(np.stack([rng.uniform(0.1, 0.9, hw), rng.uniform(0.1, 0.9, hw), np.full(hw, 0.02),
                           np.full(hw, 0.03), np.full(hw, 0.004), rng.uniform(0.2, 0.8, hw),
                           np.full(hw, 8.0), rng.uniform(0.5, 2.0, hw)], 1), dtype)
    samples = {k: dev(v) for k, v in scenes.random_samples(rng, spp, hw).items()}
    cam = scenes.top_down_camera(pixel_size=0.5)
    fld = scenes.two_lobe_field(4)
    rec = torch.from_numpy(_record_bytes(cen, dtype)).cuda()
    acc = np.zeros((hw, 8))
    for f in range(n):
        gp = GuidePass(W, H, spp=spp, gamma_dtype=dtype, seed=77, stochastic_round=1)
        gp.pg_set_gamma(rec)
        gp.pg_reproject(dev(g0), dev(g1), cam, dev(g0))
        gp.pg_sample(dev(g0), dev(g1), cam, fld, 1000 + f)     # sets the frame of the rounding bits
        gp.pg_update(dev(g0), dev(g1), cam, samples)
        acc += _records_to_central(host(gp.pg_get_gamma()), dtype)
        gp.close()
    mean = acc / n
    # the binary32 update itself, from an FP32 context (same arithmetic, no rounding)
    gp = GuidePass(W, H, spp=spp, gamma_dtype="f32", seed=77)
    set_gamma_rows(gp, _central_to_raw_moments(cen))
    gp.pg_reproject(dev(g0), dev(g1), cam, dev(g0))
    gp.pg_update(dev(g0), dev(g1), cam, samples)
    exact = _raw_to_central(get_gamma_rows(gp))
    moved = np.abs(exact - cen) > 0
    ulp = _ulp(exact, dtype)
    # standard deviation of a mean of n roundings is at most ulp / (2 sqrt n)
    err = np.abs(mean - exact)[moved] / ulp[moved]
    assert moved[:, :6].mean() > 0.5
    assert np.max(err) < 5.0 / (2 * np.sqrt(n)) + 0.02, np.max(err)
    rn_err = np.abs(_round(exact, dtype) - exact)[moved] / ulp[moved]
    assert rn_err.mean() > 5 * err.mean()


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_16_bit_store_rounds_to_nearest_and_saturates(dtype):
    """The 16-bit store of Gamma, bit for bit: round to nearest, FP16
    saturating at +-65504 (also for values that would round to infinity) and
    keeping its subnormals, BF16 unclamped. With a zero mean the stored central
    moments are the given second moments exactly, so every field of the record
    is a given binary32 value rounded once."""
    import torch
    W, H = 64, 8
    hw = W * H
    rng = np.random.default_rng(5)
    mag = np.exp(rng.uniform(np.log(1e-9), np.log(3e5), (hw, 8)))
    vals = (mag * rng.choice([-1.0, 1.0], (hw, 8))).astype(np.float32)
    vals[:, 0:2] = 0.0                                     # the mean: central = raw second moments
    vals[:8, 7] = np.float32([65504, 65519.9, 65520, 1e6, -65520, -1e9, 6e-8, 3e-5])
    par = scenes.Params(W, H)
    gp = guide(par, dtype)
    set_gamma_rows(gp, vals)
    rec = host(gp.pg_get_gamma())
    gp.close()
    t = torch.from_numpy(vals.astype(np.float32))
    if dtype == "f16":
        ref = t.clamp(-65504.0, 65504.0).to(torch.float16)
    else:
        ref = t.to(torch.bfloat16)
    assert np.array_equal(rec, ref.contiguous().view(torch.uint8).reshape(-1).numpy())
