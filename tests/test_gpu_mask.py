"""The occlusion mask keeps its relative precision where it approaches 0.
The field's radiance is L = m(x, w) times the lobes, m = (1 + sin(pi A)
cos(pi B)) / 2 with phases A, B of the shading point and the direction. The
kernels write m through the distances of its phases to their extrema, so
near a minimum (sin(pi A) cos(pi B) -> -1) the evaluation stays within a
few ulp of m itself; a product of separately rounded sine and cosine would
leave an absolute error near 6e-8, which swamps an m of 1e-10. Checked
through pg_eval at directions placed 1e-2 to 1e-5 half-turns from a minimum
of the mask, with the evaluation tolerance of the other parity tests (1e-5
relative plus 4e-7 times the value's gradient in the direction)."""
import numpy as np
import pytest

import oracle as O
from paper_2112_09728_gb300 import scenes

from _pg import close, dev, guide, host, ocam, ocfg, ofld
from test_gpu_parity import oracle_grad_norm

pytestmark = pytest.mark.gpu


def _case():
    W, H = 32, 2
    hw = W * H
    par = scenes.Params(W, H, seed=5)
    cam = scenes.top_down_camera(pixel_size=0.01)
    f1, f2, g = 1.0 / 97.0, 1.0 / 131.0, 0.5
    fld = scenes.Field(dirs=np.array([[0.0, 0.0, 1.0]]), kappas=np.array([5.0]), amps=np.array([1.0]),
                       constant=0.0, mask=(f1, f2, g))
    g0 = np.tile(np.array([[0.0, 0.0, 1.0, 2.0]], np.float32), (hw, 1))
    g1 = np.tile(np.array([[0.0, 0.0, -1.0, 0.8]], np.float32), (hw, 1))
    oc = ocam(cam)
    pos = np.array([o + 2.0 * d for o, d in (O.camera_ray(oc, W, H, i % W, i // W) for i in range(hw))])
    # a minimum of the mask: sin(pi A) = -1 (A = -1/2) and cos(pi B) = 1 (B = 0),
    # with A = 2 (f1 x + g w_x), B = 2 (f2 y + g w_y); then offsets of the phases
    rng = np.random.default_rng(3)
    off = 10.0 ** rng.uniform(-5.0, -2.0, (hw, 2)) * rng.choice([-1.0, 1.0], (hw, 2))
    wx = ((-0.5 + off[:, 0]) / 2.0 - f1 * pos[:, 0]) / g
    wy = ((0.0 + off[:, 1]) / 2.0 - f2 * pos[:, 1]) / g
    near = np.stack([wx, wy, np.sqrt(1.0 - wx * wx - wy * wy)], 1)
    far = scenes.unit_hemisphere_dirs(rng, hw, zmin=0.2)
    dirs = np.stack([near, far]).astype(np.float32)
    gam = np.tile(O.init_gamma(ocfg(par), 1)[0], (hw, 1))
    return par, cam, fld, g0, g1, gam, dirs


def test_mask_keeps_its_relative_precision_near_zero():
    par, cam, fld, g0, g1, gam, dirs = _case()
    gp = guide(par)
    out = host(gp.pg_eval(dev(g0), dev(g1), cam, fld, dev(dirs))["radiance"]).astype(np.float64)
    gp.close()
    cfg, oc, of = ocfg(par), ocam(cam), ofld(fld)
    ref = O.evaluate(cfg, oc, of, g0, g1, gam, dirs)["radiance"]
    grad = oracle_grad_norm(cfg, oc, of, g0, g1, gam, dirs)["radiance"]
    # the radiance near the minimum spans more than four decades, down to 2e-9
    assert ref[0].max() / ref[0].min() > 1e4 and ref[0].min() < 1e-8
    assert close(out, ref, 1e-5, 4e-7 * grad + 1e-30) <= 1.0
