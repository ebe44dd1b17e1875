"""Writes the FP64 ground truth I(p) = int L f_r cos dw (Eq. 1) that image
MSE is scored against, for three workloads of paper_2112_09728_gb300.scenes:

  pan_1080p_ground_truth.txt   4096 world texels of the 1920x1080 pan
                               workload, each visible in every frame 30-59
                               (at pixel (xw - 2t, yw) of frame t; the
                               orthographic view and the texel's G-buffer are
                               the same in every frame, hence so is I)
  orbit_4k_ground_truth.txt    512 fixed pixels of the 3840x2160 orbit
                               workload in each of frames 24-39 (the pinhole
                               camera moves, so I is per frame)
  diff_512_ground_truth.txt    the 512x512 differentiation workload (flat,
                               unmasked: one value for every pixel)

Every value comes from the oracle's or_ground_truth (adaptive cubature,
relative tolerance 1e-8) on the workload's own G-buffer, camera and field,
the field rounded to binary32 as the library receives it. Run from the
repository root: python tests/golden/make_ground_truth.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2112_09728_gb300 import scenes  # noqa: E402

TOL = 1e-8
PAN_FRAMES = range(30, 60)
ORBIT_FRAMES = range(24, 40)


def ofield(fld):
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    return O.make_field(f32(fld.dirs), f32(fld.kappas), f32(fld.amps), float(np.float32(fld.constant)),
                        None if fld.mask is None else [float(np.float32(m)) for m in fld.mask])


def ocamera(c):
    return O.make_camera(c.kind, c.origin, c.fwd, c.right, c.up, c.pixel_size, c.tan_half_fov)


def pan(n=4096, seed=30):
    W, H = 1920, 1080
    wl = scenes.workload_pan(W, H, frames=PAN_FRAMES.stop)
    sc, fld = wl["scene"], wl["field"]
    lo, hi = 2 * (PAN_FRAMES.stop - 1), 2 * PAN_FRAMES.start + W - 1      # visible in every frame
    rng = np.random.default_rng(seed)
    cells = rng.choice((hi - lo + 1) * H, n, replace=False)
    xw, yw = lo + cells % (hi - lo + 1), cells // (hi - lo + 1)
    t = PAN_FRAMES.start
    g0, g1, _ = sc.gbuffer(t)
    I = O.ground_truth(O.make_config(W, H), ocamera(sc.camera(t)), ofield(fld), g0, g1, xw - 2 * t, yw, tol_rel=TOL)
    with open(os.path.join(HERE, "pan_1080p_ground_truth.txt"), "w") as f:
        f.write("# FP64 ground truth I(p) = int L f_r cos dw (Eq. 1) of world texels (xw, yw) of the\n"
                "# 1920x1080 pan workload, seen at pixel (xw - 2t, yw) of frame t for t in 30..59.\n"
                "# Written by tests/golden/make_ground_truth.py (oracle or_ground_truth, tol_rel %g).\n"
                "# xw yw I\n" % TOL)
        for a, b, v in zip(xw, yw, I):
            f.write("%d %d %.17g\n" % (a, b, v))


def orbit(n=512, seed=24):
    W, H = 3840, 2160
    wl = scenes.workload_4k(W, H)
    sc, fld = wl["scene"], wl["field"]
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(W * H, n, replace=False))
    xs, ys = idx % W, idx // W
    cfg = O.make_config(W, H, spp=wl["params"].spp)
    of = ofield(fld)
    g0 = np.zeros((W * H, 4), np.float32)
    g1 = np.zeros((W * H, 4), np.float32)
    rows = []
    for t in ORBIT_FRAMES:
        a0, a1 = sc.surface_at(t, xs, ys)
        g0[idx], g1[idx] = a0, a1
        I = O.ground_truth(cfg, ocamera(sc.camera(t)), of, g0, g1, xs, ys, tol_rel=TOL)
        rows += [(t, x, y, v) for x, y, v in zip(xs, ys, I)]
    with open(os.path.join(HERE, "orbit_4k_ground_truth.txt"), "w") as f:
        f.write("# FP64 ground truth I(p) = int L f_r cos dw (Eq. 1) at 512 fixed pixels (x, y) of the\n"
                "# 3840x2160 orbit workload in frames 24..39.\n"
                "# Written by tests/golden/make_ground_truth.py (oracle or_ground_truth, tol_rel %g).\n"
                "# frame x y I\n" % TOL)
        for t, x, y, v in rows:
            f.write("%d %d %d %.17g\n" % (t, x, y, v))


def diff():
    wl = scenes.workload_diff()
    par, fld = wl["params"], wl["field"]
    g0, g1, _ = wl["gbuf"](0)
    cfg = O.make_config(par.width, par.height)
    I = O.ground_truth(cfg, ocamera(wl["camera"]), ofield(fld), g0, g1, [0, 511, 200], [0, 511, 300], tol_rel=TOL)
    assert np.ptp(I) <= 1e-12 * abs(I[0])      # every pixel sees the same integrand
    with open(os.path.join(HERE, "diff_512_ground_truth.txt"), "w") as f:
        f.write("# FP64 ground truth I(p) = int L f_r cos dw (Eq. 1) of every pixel of the 512x512\n"
                "# differentiation workload (flat Lambertian 0.8, normal +z, two vMF lobes + 0.05).\n"
                "# Written by tests/golden/make_ground_truth.py (oracle or_ground_truth, tol_rel %g).\n"
                "%.17g\n" % (TOL, I[0]))


if __name__ == "__main__":
    for name in (sys.argv[1:] or ["pan", "orbit", "diff"]):
        t0 = time.time()
        globals()[name]()
        print("%s: %.1f s" % (name, time.time() - t0), file=sys.stderr)
