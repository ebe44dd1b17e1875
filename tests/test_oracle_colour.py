"""Pins of the oracle's coloured radiance (Sec. 3.1: the EM samples are
weighted by the luminance of the radiance), on the CPU.

Luminance is linear in the colour channels, and nothing the pass decides
(strategy, draw, density, MIS) looks at the radiance. So one frame with a
coloured field must give
* the same Gamma, and the same per-sample records, as the same frame with
  the monochrome field of the luminances (Y of every lobe's colour and of
  the constant), and
* per channel, the same image as the same frame with the monochrome field of
  that channel (the image is the only thing that sees the colour).
"""
import numpy as np

import oracle as O
from paper_2112_09728_gb300 import scenes

from _pg import ocam, ocfg, ofld

Y = np.array([0.2126, 0.7152, 0.0722])


def test_coloured_frame_trains_on_luminance_and_renders_each_channel():
    W, H, spp = 24, 16, 2
    rng = np.random.default_rng(8)
    g0, g1 = scenes.random_gbuffer(rng, W, H, glass_frac=0.1)
    gam = scenes.random_gamma(rng, W * H)
    par = scenes.Params(W, H, spp=spp, seed=77, transparent=1, ggx_f0=0.3)
    cam = ocam(scenes.top_down_camera(pixel_size=0.3))
    mono = scenes.masked_lobe_field(4, n_lobes=3, kappa_hi=80.0, constant=0.05)
    col = scenes.coloured(mono, 4)
    cfg = ocfg(par)
    out_c, _, s_c, img_c = O.frame(cfg, cam, ofld(col), 2, g0, g1, g0, gam.astype(np.float64))
    assert img_c.shape == (3 * W * H,)
    # the luminance field: Y of the colours as the kernels receive them (binary32)
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    mask = [float(np.float32(m)) for m in col.mask]
    lum_o = O.make_field(f32(col.dirs), f32(col.kappas), f32(col.rgb) @ Y, float(f32(col.constant_rgb) @ Y), mask)
    out_y, _, s_y, img_y = O.frame(cfg, cam, lum_o, 2, g0, g1, g0, gam.astype(np.float64))
    assert np.allclose(out_c, out_y, rtol=1e-12, atol=1e-14)
    for k in ("radiance", "estimate", "pdf", "mis"):
        assert np.allclose(s_c[k], s_y[k], rtol=1e-12, atol=1e-15), k
    assert (s_c["strategy"] == s_y["strategy"]).all()
    # luminance of the coloured image is the luminance field's image
    assert np.allclose(img_c.reshape(3, -1).T @ Y, img_y, rtol=1e-12, atol=1e-15)
    for c in range(3):
        ch = O.make_field(f32(col.dirs), f32(col.kappas), f32(col.rgb)[:, c], float(f32(col.constant_rgb)[c]), mask)
        _, _, _, img_ch = O.frame(cfg, cam, ch, 2, g0, g1, g0, gam.astype(np.float64))
        assert np.allclose(img_c.reshape(3, -1)[c], img_ch, rtol=1e-12, atol=1e-15), c
