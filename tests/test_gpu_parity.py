"""Parity of the CUDA guide pass with the FP64 oracle on identical seeded inputs.

Tolerances (derived in the design notes):
  * integer work is bit-exact: Philox words, reprojection accept/reject and the
    previous-pixel copy, strategy choices away from their decision margins;
  * values evaluated at the SAME input (pdfs at given directions, the EM step
    from given samples) agree to 1e-5 relative plus the value's sensitivity to
    the ~2e-7 rounding of the binary32 coordinate transforms;
  * values at SAMPLED directions agree to 1e-5 relative plus the oracle's own
    gradient times the measured distance between the two sampled directions.
Samples whose decision (strategy, square edge, GGX horizon) lies within 1e-5 of
its threshold may legitimately differ; they are counted, bounded and excluded.
"""
import numpy as np
import pytest

import oracle as O
from paper_2112_09728_gb300 import scenes

from _pg import close, dev, get_gamma_rows, guide, host, ocam, ocfg, ofld, set_gamma_rows

pytestmark = pytest.mark.gpu

MARGIN = 1e-5


def _tangents(w):
    a = np.where(np.abs(w[..., :1]) < 0.9, [[1.0, 0, 0]], [[0, 1.0, 0]])
    t1 = np.cross(w, a)
    t1 /= np.linalg.norm(t1, axis=-1, keepdims=True)
    t2 = np.cross(w, t1)
    return t1, t2


def oracle_grad_norm(cfg, cam, fld, g0, g1, gam, dirs, reinit=None, h=2e-6):
    """|d v / d w| per eval key at each direction, by central differences of the
    oracle's own evaluation: two tangential directions and the radial one
    (binary32 directions are unit only to ~1.2e-7, and a vMF lobe's value
    moves by kappa times that)."""
    dirs = np.asarray(dirs, np.float64)
    t1, t2 = _tangents(dirs)
    g2 = {}
    pairs = [(dirs * np.cos(h) + t * np.sin(h), dirs * np.cos(h) - t * np.sin(h)) for t in (t1, t2)]
    pairs.append((dirs * (1 + h), dirs * (1 - h)))
    for wp, wm in pairs:
        vp = O.evaluate(cfg, cam, fld, g0, g1, gam, wp, reinit)
        vm = O.evaluate(cfg, cam, fld, g0, g1, gam, wm, reinit)
        for k in vp:
            g2[k] = g2.get(k, 0.0) + ((vp[k] - vm[k]) / (2 * h)) ** 2
    return {k: np.sqrt(v) for k, v in g2.items()}


def _scene(seed, W, H, spp=1, ggx_frac=0.5, rough_lo=0.02):
    rng = np.random.default_rng(seed)
    g0, g1 = scenes.random_gbuffer(rng, W, H, ggx_frac=ggx_frac, rough_lo=rough_lo)
    gam = scenes.random_gamma(rng, W * H)
    par = scenes.Params(W, H, spp=spp, seed=seed * 7919 + 3)
    cam = scenes.top_down_camera(pixel_size=0.37)
    fld = scenes.masked_lobe_field(seed, n_lobes=3, kappa_hi=200.0, constant=0.05)
    return rng, par, cam, fld, g0, g1, gam


# ---------------------------------------------------------------------------
def test_philox_bit_exact_and_matches_curand():
    import torch
    from paper_2112_09728_gb300.guide import pg_philox
    rng = np.random.default_rng(1)
    n = 100003
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, 2, dtype=np.uint64).astype(np.uint32)
    ref = O.philox(ctr, key)
    t = torch.from_numpy(ctr.view(np.int32)).cuda()
    own = host(pg_philox(t, key)).view(np.uint32)
    cur = host(pg_philox(t, key, use_curand=True)).view(np.uint32)
    assert (own == ref).all()
    assert (cur == ref).all()


def test_eval_matches_oracle_at_given_directions():
    W, H, n = 37, 23, 6
    rng, par, cam, fld, g0, g1, gam = _scene(2, W, H)
    dirs = scenes.random_directions(rng, n, W * H)
    gp = guide(par)
    set_gamma_rows(gp, gam)
    out = {k: host(v).astype(np.float64) for k, v in gp.pg_eval(dev(g0), dev(g1), cam, fld, dev(dirs)).items()}
    cfg, oc, of = ocfg(par), ocam(cam), ofld(fld)
    g64 = gam.astype(np.float64)
    ref = O.evaluate(cfg, oc, of, g0, g1, g64, dirs)
    grad = oracle_grad_norm(cfg, oc, of, g0, g1, g64, dirs)
    for k in ref:
        # pdfs: relative to the mixture they enter; MIS weights live in [0, 1]
        scale = np.abs(ref["pmix"]) if k in ("pg", "pb", "pmix") else (1.0 if k.startswith("w_") else 0.0)
        atol = 1e-6 * scale + 4e-7 * grad[k] + 1e-30
        worst = close(out[k], ref[k], 1e-5, atol)
        if worst > 1.0:
            r = np.abs(out[k] - ref[k]) / (1e-5 * np.abs(ref[k]) + atol)
            s_, i_ = np.unravel_index(np.argmax(r), r.shape)
            print(k, "dir", s_, "pixel", i_, "gpu", out[k][s_, i_], "oracle", ref[k][s_, i_], "grad",
                  grad[k][s_, i_], "g1", g1[i_], "g0", g0[i_], "w", dirs[s_, i_],
                  {kk: (out[kk][s_, i_], ref[kk][s_, i_]) for kk in ref})
        assert worst <= 1.0, (k, worst)


def test_reproject_matches_oracle():
    W, H = 41, 29
    hw = W * H
    rng = np.random.default_rng(3)
    # gently tilted previous normals (any two within 0.3 rad pass the 0.9 test)
    g0p, g1 = scenes.random_gbuffer(rng, W, H, max_tilt=0.15)
    g0p[:, 3] = rng.uniform(5.0, 5.2, hw).astype(np.float32)   # a smooth depth
    g0 = g0p.copy()
    # motion: integer, fractional, off-screen, NaN
    mv = rng.choice([-2.0, 0.0, 1.0, 3.0], (hw, 2)).astype(np.float32)
    frac = rng.random(hw) < 0.3
    mv[frac] = rng.uniform(-4, 4, (frac.sum(), 2)).astype(np.float32)
    off = rng.random(hw) < 0.05
    mv[off, 0] = np.float32(W + 5)
    mv[rng.random(hw) < 0.01, 1] = np.nan
    g1[:, :2] = mv
    # depth jumps around the 10 % threshold, new normals (small and large tilts)
    j = rng.random(hw) < 0.2
    g0[j, 3] *= rng.uniform(0.85, 1.15, j.sum()).astype(np.float32)
    t = rng.random(hw) < 0.3
    g0[t, :3] = scenes.random_normals(rng, int(t.sum()), 0.6)
    gam = scenes.random_gamma(rng, hw)
    par = scenes.Params(W, H)
    gp = guide(par)
    set_gamma_rows(gp, gam)
    import torch
    acc = torch.empty(hw, dtype=torch.uint8, device="cuda")
    gp.pg_reproject(dev(g0), dev(g1), scenes.top_down_camera(), dev(g0p), acc)
    from paper_2112_09728_gb300.guide import planes_to_rows
    got = host(planes_to_rows(gp.pg_get_reprojected())).astype(np.float64)
    ref, racc, q = O.reproject(ocfg(par), g0, g1, g0p, gam.astype(np.float64))
    acc = host(acc)
    assert (acc == racc).all()
    assert 0.3 < racc.mean() < 0.95
    same = np.zeros(hw, bool)
    same[racc == 1] = (g0p[q[racc == 1], :3] == g0[racc == 1, :3]).all(1)
    assert (got[same] == ref[same]).all()                      # plain copies: bit-exact
    fc = (racc == 1) & ~same
    assert fc.sum() > 20
    assert close(got[fc], ref[fc], 1e-5, 2e-6) <= 1.0           # frame change
    rej = racc == 0
    assert (got[rej, 6] == -1).all() and (ref[rej, 6] == 0).all()
    assert close(got[rej][:, [0, 1, 2, 3, 4, 5, 7]], ref[rej][:, [0, 1, 2, 3, 4, 5, 7]], 1e-7, 1e-30) <= 1.0


def _sample_both(seed, W, H, spp, gamma_dtype="f32"):
    import torch
    from paper_2112_09728_gb300.guide import alloc_samples
    rng, par, cam, fld, g0, g1, gam = _scene(seed, W, H, spp=spp)
    gp = guide(par, gamma_dtype)
    set_gamma_rows(gp, gam)
    gp.pg_reproject(dev(g0), dev(g1), cam, dev(g0))
    s = alloc_samples(spp, W * H)
    img = torch.empty(W * H, device="cuda")
    gp.pg_sample(dev(g0), dev(g1), cam, fld, 5, s, img)
    got = {k: host(v) for k, v in s.items()}
    cfg, oc, of = ocfg(par), ocam(cam), ofld(fld)
    ref, rimg = O.sample(cfg, oc, of, 5, g0, g1, gam.astype(np.float64))
    return dict(gp=gp, got=got, img=host(img), ref=ref, rimg=rimg, cfg=cfg, oc=oc, of=of, g0=g0, g1=g1,
                gam=gam, par=par, cam=cam, fld=fld, spp=spp, hw=W * H)


def test_sample_matches_oracle():
    S = _sample_both(4, 33, 17, 4)
    got, ref, spp, hw = S["got"], S["ref"], S["spp"], S["hw"]
    amb = ref["margin"] < MARGIN
    assert amb.mean() < 2e-3
    ok = ~amb
    assert (got["strategy"][ok] == ref["strategy"][ok]).all()
    st = ref["strategy"][ok] & 3
    assert (st == 1).mean() > 0.2 and (st == 0).mean() > 0.2 and (st == 2).any()
    wg = np.stack([got["wx"], got["wy"], got["wz"]], -1).astype(np.float64)
    wr = np.stack([ref["wx"], ref["wy"], ref["wz"]], -1)
    dw = np.linalg.norm(wg - wr, axis=-1)
    assert dw[ok].max() < 2e-6
    valid = ok & ((ref["strategy"] & 4) == 0)
    grad = oracle_grad_norm(S["cfg"], S["oc"], S["of"], S["g0"], S["g1"], S["gam"].astype(np.float64),
                            wr.reshape(spp, hw, 3))
    gF = {k: v.reshape(-1) for k, v in grad.items()}
    dwv = np.maximum(dw, 4e-7)
    assert close(got["pdf"][valid], ref["pdf"][valid], 1e-5, (2 * gF["pmix"] * dwv)[valid]) <= 1.0
    assert close(got["radiance"][valid], ref["radiance"][valid], 1e-5, (2 * gF["radiance"] * dwv)[valid]) <= 1.0
    # F = fcos / pmix: first-order bound from the two gradients
    F = ref["estimate"]
    gradF = (gF["fcos"] + np.abs(F) * gF["pmix"]) / np.maximum(ref["pdf"], 1e-30)
    assert close(got["estimate"][valid], F[valid], 2e-5, (2 * gradF * dwv)[valid] + 1e-12) <= 1.0
    assert close(got["mis"][valid], ref["mis"][valid], 2e-5, (2 * (gF["pmix"] / np.maximum(ref["pdf"], 1e-30))
                                                            * dwv)[valid] + 1e-7) <= 1.0
    # the pixel estimate, on pixels with no ambiguous sample
    pix_ok = ~amb.reshape(spp, hw).any(0)
    tolF = (2 * gradF * dwv + 2e-5 * np.abs(F)).reshape(spp, hw).sum(0) / spp
    assert close(S["img"][pix_ok], S["rimg"][pix_ok], 0, tolF[pix_ok] + 1e-12) <= 1.0


def test_update_matches_oracle_from_given_samples():
    W, H, spp = 29, 19, 3
    rng, par, cam, fld, g0, g1, gam = _scene(5, W, H, spp=spp)
    samples = scenes.random_samples(rng, spp, W * H)
    gp = guide(par)
    set_gamma_rows(gp, gam)
    gp.pg_reproject(dev(g0), dev(g1), cam, dev(g0))
    gp.pg_update(dev(g0), dev(g1), cam, {k: dev(v) for k, v in samples.items()})
    got = get_gamma_rows(gp)
    ref = O.update(ocfg(par), ocam(cam), g0, g1, gam.astype(np.float64),
                   {k: (v.astype(np.float64) if v.dtype != np.uint8 else v) for k, v in samples.items()})
    assert (got[:, 6] == ref[:, 6]).all()            # epoch counter: exact
    changed = np.abs(ref[:, :5] - gam[:, :5]).max(1) > 0
    assert changed.mean() > 0.3
    assert close(got[:, :5], ref[:, :5], 1e-5, 1e-6) <= 1.0
    assert close(got[:, 5], ref[:, 5], 1e-5, 1e-6) <= 1.0
    assert close(got[:, 7], ref[:, 7], 1e-5, 1e-6) <= 1.0


def _frame_both(seed, W, H, spp, frame=3):
    import torch
    rng, par, cam, fld, g0, g1, gam = _scene(seed, W, H, spp=spp)
    gp = guide(par)
    set_gamma_rows(gp, gam)
    img = torch.empty(W * H, device="cuda")
    gp.pg_frame(dev(g0), dev(g1), cam, dev(g0), fld, frame, img)
    gp.pg_check()
    got = get_gamma_rows(gp)
    ref, acc, s, rimg = O.frame(ocfg(par), ocam(cam), ofld(fld), frame, g0, g1, g0, gam.astype(np.float64))
    return got, host(img), ref, rimg, s, gam


def test_fused_frame_matches_oracle():
    W, H, spp = 45, 31, 2
    got, img, ref, rimg, s, gam = _frame_both(6, W, H, spp)
    amb = (s["margin"] < MARGIN).reshape(spp, -1).any(0)
    assert amb.mean() < 5e-3
    ok = ~amb
    assert (got[ok, 6] == ref[ok, 6]).all()
    assert close(got[ok, :5], ref[ok, :5], 1e-5, 2e-6) <= 1.0
    assert close(got[ok, 5], ref[ok, 5], 1e-5, 5e-6) <= 1.0
    assert close(got[ok, 7], ref[ok, 7], 1e-4, 1e-6) <= 1.0
    assert close(img[ok], rimg[ok], 1e-4, 1e-6) <= 1.0


def test_staged_equals_fused_on_gpu():
    import torch
    from paper_2112_09728_gb300.guide import alloc_samples
    W, H, spp = 50, 22, 3
    rng, par, cam, fld, g0, g1, gam = _scene(7, W, H, spp=spp)
    a, b = guide(par), guide(par)
    set_gamma_rows(a, gam)
    set_gamma_rows(b, gam)
    ia, ib = torch.empty(W * H, device="cuda"), torch.empty(W * H, device="cuda")
    a.pg_frame(dev(g0), dev(g1), cam, dev(g0), fld, 9, ia)
    b.pg_reproject(dev(g0), dev(g1), cam, dev(g0))
    s = alloc_samples(spp, W * H)
    b.pg_sample(dev(g0), dev(g1), cam, fld, 9, s, ib)
    b.pg_update(dev(g0), dev(g1), cam, s)
    # the two paths run the same device functions, but nvcc may contract
    # multiply-adds differently per kernel, so agreement is to rounding
    assert close(host(ib), host(ia), 1e-6, 1e-9) <= 1.0
    assert close(get_gamma_rows(b), get_gamma_rows(a), 1e-5, 1e-6) <= 1.0


def test_small_workload_eight_frames_free_running():
    """64x64, 1 spp, 8 frames, static camera, flat Lambertian, two lobes: the
    GPU and the oracle each run their own state forward."""
    import torch
    wl = scenes.workload_small()
    par, cam, fld = wl["params"], wl["camera"], wl["field"]
    gp = guide(par)
    cfg, oc, of = ocfg(par), ocam(cam), ofld(fld)
    g0, g1, g0p = wl["gbuf"](0)
    gref = O.init_gamma(cfg, par.width * par.height, pi=par.init_pi)
    img = torch.empty(par.width * par.height, device="cuda")
    amb = np.zeros(par.width * par.height, bool)
    for t in range(wl["frames"]):
        gp.pg_frame(dev(g0), dev(g1), cam, dev(g0p), fld, t, img)
        gref, acc, s, rimg = O.frame(cfg, oc, of, t, g0, g1, g0p, gref)
        amb |= (s["margin"] < MARGIN).reshape(par.spp, -1).any(0)
        assert acc.all()
        ok = ~amb
        assert close(host(img)[ok], rimg[ok], 2e-4, 1e-6) <= 1.0
    gp.pg_check()
    got = get_gamma_rows(gp)
    ok = ~amb
    assert ok.mean() > 0.98
    assert (got[ok, 6] == gref[ok, 6]).all()
    assert close(got[ok, :6], gref[ok, :6], 1e-4, 2e-6) <= 1.0


def test_pan_workload_reprojection_and_parity():
    """The panning heightfield workload at a reduced 96x40: the two newly
    exposed columns are re-initialised every frame, everything else is a
    shifted copy plus one EM step."""
    import torch
    wl = scenes.workload_pan(96, 40, frames=5)
    par, fld = wl["params"], wl["field"]
    gp = guide(par)
    cfg, of = ocfg(par), ofld(fld)
    gref = O.init_gamma(cfg, par.width * par.height, pi=par.init_pi)
    img = torch.empty(par.width * par.height, device="cuda")
    amb = np.zeros(par.width * par.height, bool)
    for t in range(wl["frames"]):
        g0, g1, g0p = wl["gbuf"](t)
        cam = wl["camera"](t)
        acc = torch.empty(par.width * par.height, dtype=torch.uint8, device="cuda")
        # the staged reprojection exposes the accept mask
        gp.pg_reproject(dev(g0), dev(g1), cam, dev(g0p), acc)
        a = host(acc).reshape(par.height, par.width)
        assert a[:, :-2].all() and not a[:, -2:].any()
        from paper_2112_09728_gb300.guide import alloc_samples
        s = alloc_samples(par.spp, par.width * par.height)
        gp.pg_sample(dev(g0), dev(g1), cam, fld, t, s, img)
        gp.pg_update(dev(g0), dev(g1), cam, s)
        gref, racc, rs, rimg = O.frame(cfg, ocam(cam), of, t, g0, g1, g0p, gref)
        assert (racc.reshape(par.height, par.width) == a).all()
        amb |= (rs["margin"] < MARGIN).reshape(par.spp, -1).any(0)
        # an ambiguity at pixel p travels left with the camera: exclude the row tail
        amb_shift = amb.reshape(par.height, par.width)
        amb = np.concatenate([amb_shift[:, 2:], np.zeros((par.height, 2), bool)], 1).reshape(-1) | amb
    got = get_gamma_rows(gp)
    ok = ~amb
    assert ok.mean() > 0.9
    assert (got[ok, 6] == gref[ok, 6]).all()
    assert close(got[ok, :6], gref[ok, :6], 1e-4, 2e-6) <= 1.0
