"""Pins of the oracle's neighbour-VPL reuse (Sec. 3.2, Sec. 4.2), on the CPU.

* The pick law: N = 5 + floor(15 (kMax - k) / kMax) capped at the number of
  candidates, distinct candidates from the window, never the pixel itself,
  every candidate equally likely over pixels.
* Exact statistics: equal Lambertian pixels under a constant field, every
  pixel re-initialised (guide off, all draws from the BRDF): each VPL weighs
  exactly L0 * albedo, so the frame's mass W is L0 * albedo times one plus the
  number of picks that fall inside the image.
* Unbiasedness across tilted neighbours: on a checkerboard of two normals the
  expected mass of an interior pixel is its own integral of L f_r cos plus,
  per neighbour, the integral of L f_r cos over the directions the
  neighbour's cosine lobe reaches. A weight taken with the receiving pixel's
  own BRDF density instead of the source's would converge to a different
  value, which the test computes too and keeps well away from.
"""
import math

import numpy as np

import oracle as O
from paper_2112_09728_gb300 import scenes

from _pg import ocam


def _cfg(W, H, R, spp=1, k_max=32, seed=5):
    return O.make_config(W, H, spp=spp, seed=seed, k_max=k_max, reuse_radius=R)


def test_pick_law_counts_window_and_distinctness():
    for R, spp, k_max in ((1, 1, 32), (2, 1, 32), (2, 3, 16), (3, 1, 32)):
        c = _cfg(40, 30, R, spp, k_max)
        cand = ((2 * R + 1) ** 2 - 1) * spp
        for k in (0, 1, k_max // 2, k_max - 1, k_max, k_max + 5, -1):
            kc = min(max(k, 0), k_max)
            want = min(5 + (15 * (k_max - kc)) // k_max, cand)
            for pix in (0, 17, 1199):
                dx, dy, sm = O.reuse_picks(c, k, pix, 3)
                assert len(dx) == want
                assert (np.abs(dx) <= R).all() and (np.abs(dy) <= R).all()
                assert not ((dx == 0) & (dy == 0)).any()
                assert ((sm >= 0) & (sm < spp)).all()
                assert len(set(zip(dx.tolist(), dy.tolist(), sm.tolist()))) == want


def test_pick_law_offsets_are_uniform_over_pixels():
    R = 2
    c = _cfg(64, 64, R)
    counts = {}
    n_pix = 12000
    for pix in range(n_pix):
        dx, dy, _ = O.reuse_picks(c, 32, pix, 11)      # N = 5
        for a, b in zip(dx.tolist(), dy.tolist()):
            counts[(a, b)] = counts.get((a, b), 0) + 1
    assert len(counts) == 24
    e = n_pix * 5 / 24
    chi2 = sum((v - e) ** 2 / e for v in counts.values())
    assert chi2 < 60.0      # 23 degrees of freedom: P(chi2 > 60) < 1e-4


def _flat(W, H, normals, albedo=0.8, depth=5.0):
    g0 = np.zeros((W * H, 4), np.float32)
    g0[:, :3] = normals
    g0[:, 3] = depth
    g1 = np.zeros((W * H, 4), np.float32)
    g1[:, 2] = -1.0
    g1[:, 3] = albedo
    g0p = g0.copy()
    g0p[:, 3] = 10 * depth          # every pixel fails the depth test: re-initialised
    return g0, g1, g0p


def test_constant_field_gives_exact_mass_with_reuse():
    W, H, R = 12, 9, 2
    c = _cfg(W, H, R)
    cam = ocam(scenes.top_down_camera())
    L0 = 0.7
    fld = O.make_field(np.zeros((0, 3)), np.zeros(0), np.zeros(0), L0)
    nz = np.tile(np.array([[0, 0, 1]], np.float32), (W * H, 1))
    g0, g1, g0p = _flat(W, H, nz)
    gam = O.init_gamma(c, W * H)
    out, acc, s, _ = O.frame(c, cam, fld, 4, g0, g1, g0p, gam)
    assert (acc == 0).all() and (s["strategy"] == 0).all()
    a32 = float(np.float32(0.8))        # the albedo as the G-buffer stores it
    for i in range(W * H):
        x, y = i % W, i // W
        dx, dy, _ = O.reuse_picks(c, 0, i, 4)
        inside = ((x + dx >= 0) & (x + dx < W) & (y + dy >= 0) & (y + dy < H)).sum()
        assert abs(out[i, 7] - L0 * a32 * (1 + inside)) <= 1e-12 * L0 * (1 + inside), i
    # the guide is off on re-initialised pixels: no responsibility, mean kept
    assert np.allclose(out[:, :2], 0.5) and (out[:, 6] == 1.0).all()
    # without reuse the mass is the pixel's own draw only
    c0 = _cfg(W, H, 0)
    out0, _, _, _ = O.frame(c0, cam, fld, 4, g0, g1, g0p, gam)
    assert np.allclose(out0[:, 7], L0 * a32, rtol=1e-12)


def _sphere_grid(n_t=300, n_p=600):
    t = (np.arange(n_t) + 0.5) * math.pi / n_t
    p = (np.arange(n_p) + 0.5) * 2 * math.pi / n_p
    T, P = np.meshgrid(t, p, indexing="ij")
    w = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    dA = (np.sin(T) * (math.pi / n_t) * (2 * math.pi / n_p)).ravel()
    return w, dA


def test_reused_weights_are_unbiased_across_tilted_neighbours():
    W = H = 24
    R, albedo, beta = 1, 0.8, 0.5
    c = _cfg(W, H, R, seed=77)
    cam = ocam(scenes.top_down_camera())
    # a broad lobe on the side the tilted normal leans to, far from both
    # horizons (where a reused weight f_p / p_src grows without bound)
    fdir = np.array([[0.0, -math.sin(1.0), math.cos(1.0)]])
    fld = O.make_field(fdir, np.array([3.0]), np.array([1.0]), 0.0)
    nA = np.array([0.0, 0.0, 1.0])
    nB = np.array([0.0, -math.sin(beta), math.cos(beta)])
    xs, ys = np.meshgrid(np.arange(W), np.arange(H))
    cls = ((xs + ys) % 2).ravel()
    normals = np.where(cls[:, None] == 0, nA, nB).astype(np.float32)
    normals /= np.linalg.norm(normals, axis=1, keepdims=True)
    g0, g1, g0p = _flat(W, H, normals, albedo)
    gam = O.init_gamma(c, W * H)

    # expected masses by quadrature of the radiance field over the sphere
    w, dA = _sphere_grid()
    L = np.array([O.radiance(fld, np.zeros(3), v) for v in w])
    n32 = [normals[0].astype(np.float64), normals[1].astype(np.float64)]
    cos = [np.maximum(w @ n, 0.0) for n in n32]

    def integral(recv, src, own_density):
        both = (cos[recv] > 0) & (cos[src] > 0)
        weight = cos[src] if own_density else cos[recv]
        return float((L * albedo / math.pi * weight * both * dA).sum())

    interior = ((xs >= 1) & (xs < W - 1) & (ys >= 1) & (ys < H - 1)).ravel()
    sums = np.zeros(2)
    cnt = np.zeros(2)
    for f in range(200):
        out, _, _, _ = O.frame(c, cam, fld, 1000 + f, g0, g1, g0p, gam)
        for k in (0, 1):
            sel = interior & (cls == k)
            sums[k] += out[sel, 7].sum()
            cnt[k] += sel.sum()
    for k in (0, 1):
        o = 1 - k
        right = 5 * integral(k, k, False) + 4 * integral(k, o, False)
        wrong = 5 * integral(k, k, False) + 4 * integral(k, o, True)
        got = sums[k] / cnt[k]
        # ~0.4% standard error from 200 frames of ~240 pixels per class
        assert abs(got - right) < 0.015 * right, (k, got, right, wrong)
        assert abs(wrong - right) > 0.10 * right, (k, right, wrong)
