"""The bounds-checked build (libpg_bounds.so): every index that depends on
the data (the reprojected pixel from the motion vectors, a reused neighbour's
sample from the picks) is checked against its buffer before the access, and a
violation is reported by pg_check as PG_ERR_BOUNDS with the access skipped.

Hostile inputs are run through it first: motion vectors that are NaN, +-inf,
+-1e30, -0.0, or land exactly on and just beside the screen's edges; neighbour
reuse with windows larger than the screen (R = 8 on a 3x2 screen), several
sample counts and odd sizes; the staged frame with its accept mask. It must
report nothing. Only then do the same inputs run through the normal build,
whose results must be bit-identical (the checks change no arithmetic).
"""
import dataclasses

import numpy as np
import pytest

from paper_2112_09728_gb300 import scenes

from _pg import dev, guide, set_gamma_rows

pytestmark = pytest.mark.gpu


def _hostile_mv(rng, W, H, g1):
    """Motion vectors of every hostile kind, cycled over the pixels."""
    g1 = g1.copy()
    x = np.tile(np.arange(W), H).astype(np.float64)
    y = np.repeat(np.arange(H), W).astype(np.float64)
    f32 = lambda a: np.asarray(a, np.float32)
    kinds = [
        (np.nan, 0.0), (0.0, np.nan), (np.inf, 0.0), (-np.inf, 0.0), (0.0, np.inf), (0.0, -np.inf),
        (1e30, 0.0), (-1e30, 0.0), (0.0, 1e30), (0.0, -1e30), (-0.0, -0.0),
        (W - x - 0.5, 0.0),                                # lands exactly on the right edge (rejected)
        (W - x - 0.5 - 1e-3, 0.0),                         # just inside the last column
        (-x - 0.5, 0.0),                                   # lands exactly on the left edge (accepted)
        (-x - 0.5 - 1e-3, 0.0),                            # just outside
        (0.0, H - y - 0.5), (0.0, -y - 0.5), (0.0, -y - 0.5 - 1e-3),
        (rng.uniform(-3, 3, W * H), rng.uniform(-3, 3, W * H)),
    ]
    k = np.arange(W * H) % len(kinds)
    for j, (mx, my) in enumerate(kinds):
        sel = k == j
        g1[sel, 0] = f32(np.broadcast_to(mx, (W * H,)))[sel]
        g1[sel, 1] = f32(np.broadcast_to(my, (W * H,)))[sel]
    return g1


def _run(par, gam, g0, g1, cam, fld, bounds_check, frames=2, staged=False, dtype="f16"):
    import torch
    from paper_2112_09728_gb300.guide import alloc_samples
    gp = guide(par, gamma_dtype=dtype, bounds_check=bounds_check)
    set_gamma_rows(gp, gam)
    hw = par.width * par.height
    outs = []
    for t in range(frames):
        img = torch.empty(gp.image_planes(fld) * hw, device="cuda")
        if staged:
            acc = torch.empty(hw, dtype=torch.uint8, device="cuda")
            gp.pg_reproject(dev(g0), dev(g1), cam, dev(g0), acc)
            smp = alloc_samples(par.spp, hw)
            gp.pg_sample(dev(g0), dev(g1), cam, fld, t, smp, img)
            gp.pg_update(dev(g0), dev(g1), cam, smp)
            outs.append(acc.clone())
        else:
            gp.pg_frame(dev(g0), dev(g1), cam, dev(g0), fld, t, img)
        gp.pg_check()                         # raises on PG_ERR_BOUNDS (and PG_ERR_NUMERIC)
        outs += [img.clone(), gp.pg_get_gamma().clone()]
    gp.close()
    return outs


CASES = [
    # (W, H, spp, reuse_radius, transparent, coloured, staged)
    (45, 31, 1, 0, 0, False, False),
    (45, 31, 3, 0, 1, True, False),
    (40, 27, 2, 0, 0, False, True),
    (33, 17, 1, 2, 0, False, False),
    (33, 17, 3, 3, 1, True, False),
    (3, 2, 1, 8, 0, False, False),
    (3, 2, 5, 8, 0, False, False),
    (1, 1, 2, 1, 0, False, False),
    (257, 1, 1, 4, 0, False, False),
]


@pytest.mark.parametrize("W,H,spp,R,glass,rgb,staged", CASES)
def test_bounds_checked_build_reports_nothing_and_matches(W, H, spp, R, glass, rgb, staged):
    import torch
    rng = np.random.default_rng(W * 1000 + H * 10 + spp + R)
    g0, g1 = scenes.random_gbuffer(rng, W, H, rough_lo=0.05, glass_frac=0.1 if glass else 0.0)
    g1 = _hostile_mv(rng, W, H, g1)
    gam = scenes.random_gamma(rng, W * H)
    par = dataclasses.replace(scenes.Params(W, H, spp=spp, seed=W + H + spp), reuse_radius=R, transparent=glass)
    cam = scenes.top_down_camera(pixel_size=0.4)
    fld = scenes.masked_lobe_field(3, n_lobes=3, kappa_hi=100.0, constant=0.05)
    if rgb:
        fld = scenes.coloured(fld, 5)
    checked = _run(par, gam, g0, g1, cam, fld, True, staged=staged)
    normal = _run(par, gam, g0, g1, cam, fld, False, staged=staged)
    for a, b in zip(checked, normal):
        assert torch.equal(a, b)
