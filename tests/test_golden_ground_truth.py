"""The stored ground truth that the benchmark scores image MSE against
(tests/golden/*_ground_truth.txt, written by tests/golden/make_ground_truth.py
from the oracle's cubature of Eq. 1) is what that script computes: entries
drawn at random are recomputed here, and the files cover what the benchmark
reads (the pan's texels stay on screen in frames 30-59, the orbit's pixels
are on its screen in frames 24-39)."""
import os
import sys

import numpy as np

import oracle as O
from paper_2112_09728_gb300 import scenes

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_ground_truth as M  # noqa: E402


def _rows(name):
    return np.array([l.split() for l in open(os.path.join(HERE, "golden", name)) if not l.startswith("#")],
                    np.float64)


def test_pan_ground_truth_recomputes_and_stays_on_screen():
    r = _rows("pan_1080p_ground_truth.txt")
    assert len(r) == 4096 and len(np.unique(r[:, 1] * 4000 + r[:, 0])) == 4096
    for t in M.PAN_FRAMES:
        x = r[:, 0] - 2 * t
        assert (x >= 0).all() and (x < 1920).all()
    wl = scenes.workload_pan(1920, 1080, frames=60)
    sc = wl["scene"]
    pick = np.random.default_rng(1).choice(len(r), 12, replace=False)
    for t in (30, 59):                      # the texel's integral is the same in every frame
        g0, g1, _ = sc.gbuffer(t)
        xs, ys = (r[pick, 0] - 2 * t).astype(np.int32), r[pick, 1].astype(np.int32)
        I = O.ground_truth(O.make_config(1920, 1080), M.ocamera(sc.camera(t)), M.ofield(wl["field"]), g0, g1,
                           xs, ys, tol_rel=M.TOL)
        assert np.allclose(I, r[pick, 2], rtol=1e-12, atol=0)


def test_orbit_ground_truth_recomputes():
    r = _rows("orbit_4k_ground_truth.txt")
    assert sorted(set(r[:, 0].astype(int))) == list(M.ORBIT_FRAMES)
    assert (r[:, 1] < 3840).all() and (r[:, 2] < 2160).all()
    wl = scenes.workload_4k()
    sc = wl["scene"]
    pick = np.random.default_rng(2).choice(len(r), 8, replace=False)
    W, H = 3840, 2160
    for k in pick:
        t, x, y = int(r[k, 0]), int(r[k, 1]), int(r[k, 2])
        a0, a1 = sc.surface_at(t, [x], [y])
        g0 = np.zeros((W * H, 4), np.float32)
        g1 = np.zeros((W * H, 4), np.float32)
        g0[y * W + x], g1[y * W + x] = a0[0], a1[0]
        I = O.ground_truth(O.make_config(W, H, spp=4), M.ocamera(sc.camera(t)), M.ofield(wl["field"]), g0, g1,
                           [x], [y], tol_rel=M.TOL)
        assert np.allclose(I, r[k, 3], rtol=1e-12, atol=0)


def test_diff_ground_truth_recomputes():
    v = _rows("diff_512_ground_truth.txt").reshape(-1)
    wl = scenes.workload_diff()
    g0, g1, _ = wl["gbuf"](0)
    I = O.ground_truth(O.make_config(512, 512), M.ocamera(wl["camera"]), M.ofield(wl["field"]), g0, g1, [7], [9],
                       tol_rel=M.TOL)
    assert np.allclose(I, v, rtol=1e-12, atol=0)
