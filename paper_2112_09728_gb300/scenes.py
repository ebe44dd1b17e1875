"""Seeded synthetic inputs for the guide pass: G-buffers, cameras, radiance
fields, guide states and sample sets.

These stand in for the paper's rasterised G-buffer and its Falcor scenes
(Bistro, Sponza, San Miguel), which are not available; the traced incident
radiance is replaced by an analytic field of von Mises-Fisher lobes. The module
holds none of the guide pass's arithmetic: it only draws inputs (numpy, CPU),
which the tests feed both to the CUDA path and to the oracle.

Layouts (all float32, one row per pixel, row-major y*W + x):
  g0 [H*W, 4]  normal x, y, z, depth (distance along the primary ray)
  g1 [H*W, 4]  motion x, y (previous minus current screen position, pixels),
               roughness (negative = Lambertian), albedo
  gamma [H*W, 8]  E[X], E[Y], E[X^2], E[Y^2], E[XY], pi, k, W
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 2112097280


@dataclasses.dataclass
class Camera:
    kind: int                  # 0 orthographic, 1 pinhole
    origin: tuple
    fwd: tuple
    right: tuple
    up: tuple
    pixel_size: float = 1.0    # orthographic: world units per pixel
    tan_half_fov: float = 0.0  # pinhole: tan(vertical fov / 2)


@dataclasses.dataclass
class Field:
    dirs: np.ndarray           # [n, 3] unit directions
    kappas: np.ndarray         # [n]
    amps: np.ndarray           # [n]
    constant: float = 0.0
    mask: tuple | None = None  # (f1, f2, g) of the sinusoidal occlusion mask
    rgb: np.ndarray | None = None       # [n, 3] lobe colours (a coloured field; amps unused)
    constant_rgb: tuple | None = None   # the constant's colour (with rgb)


@dataclasses.dataclass
class Params:
    width: int
    height: int
    spp: int = 1
    seed: int = 0
    k_max: int = 32
    pi_min: float = 0.05
    pi_max: float = 0.95
    pi_reinit: float = 0.05
    depth_tol: float = 0.1
    normal_tol: float = 0.9
    rough_min: float = 0.1
    sigma2_min: float = 1e-4
    rho_max: float = 0.9
    init_mu: tuple = (0.5, 0.5)
    init_sigma: tuple = (0.1, 0.1, 0.0)
    init_pi: float = 0.5
    reuse_radius: int = 0      # neighbour-VPL reuse window radius (0: off)
    ggx_f0: float = 1.0        # Schlick reflectance of GGX at normal incidence (1: no Fresnel)
    transparent: int = 0       # 1: roughness codes <= -1.5 are transparent (else Lambertian)


def unit_hemisphere_dirs(rng, n, zmin=0.0):
    """Uniform directions on the upper hemisphere (z > zmin)."""
    z = rng.uniform(zmin, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def top_down_camera(x0=0.0, y0=0.0, height=100.0, pixel_size=1.0):
    return Camera(0, (x0, y0, height), (0.0, 0.0, -1.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0),
                  pixel_size=pixel_size)


# ----------------------------------------------------------------------------
# Workload 1: 64x64, static top-down camera, flat Lambertian, 2 lobes + 0.05.
# ----------------------------------------------------------------------------
def flat_scene(width=64, height=64, albedo=0.8, depth=1.0):
    g0 = np.zeros((height * width, 4), np.float32)
    g0[:, 2] = 1.0
    g0[:, 3] = depth
    g1 = np.zeros((height * width, 4), np.float32)
    g1[:, 2] = -1.0
    g1[:, 3] = albedo
    return g0, g1


def two_lobe_field(seed):
    rng = np.random.default_rng(seed)
    return Field(dirs=unit_hemisphere_dirs(rng, 2, zmin=0.1), kappas=np.array([20.0, 80.0]),
                 amps=np.ones(2), constant=0.05)


def workload_small(width=64, height=64, spp=1, frames=8):
    """Plain FP32 guide pass on a 64x64 screen, static camera (zero motion),
    normals +z, Lambertian albedo 0.8, two normalised vMF lobes (kappa 20 and
    80, directions drawn from the seed) plus a constant 0.05; the guide starts
    at mu = (0.5, 0.5), Sigma = 0.1 I, pi = 0.5."""
    seed = SEED_BASE + 1
    g0, g1 = flat_scene(width, height)
    return dict(params=Params(width, height, spp=spp, seed=seed), camera=top_down_camera(
        pixel_size=1.0 / width), field=two_lobe_field(seed), frames=frames,
        gbuf=lambda t: (g0, g1, g0))


def workload_diff(width=512, height=512, spp=64, steps=20):
    """The 64x64 workload's scene (flat Lambertian 0.8, the same two lobes +
    0.05) and initial guide on a 512x512 screen, 64 samples per pixel per
    step: 20 gradient steps (projected Adam, lr 1e-2) on the second-moment
    loss against 20 EM steps, each step on fresh samples."""
    seed = SEED_BASE + 4
    g0, g1 = flat_scene(width, height)
    return dict(params=Params(width, height, spp=spp, seed=seed), camera=top_down_camera(
        pixel_size=1.0 / width), field=two_lobe_field(SEED_BASE + 1), steps=steps,
        gbuf=lambda t: (g0, g1, g0))


# ----------------------------------------------------------------------------
# Workload 2: 1920x1080 pan over a heightfield, mixed Lambertian / GGX.
# ----------------------------------------------------------------------------
class Heightfield:
    """Spectral fBm: six octaves of four plane waves each, amplitude halving and
    frequency doubling per octave; heights and analytic gradients in pixel
    units of the world texel grid."""

    def __init__(self, seed, amplitude=2.0, period=256.0, octaves=6, waves=4):
        rng = np.random.default_rng(seed)
        self.terms = []
        for o in range(octaves):
            f = 2.0 * np.pi / period * 2.0 ** o
            a = amplitude * 0.5 ** o
            for _ in range(waves):
                th = rng.uniform(0, 2 * np.pi)
                self.terms.append((a, f * np.cos(th), f * np.sin(th), rng.uniform(0, 2 * np.pi)))

    def eval(self, X, Y):
        h = np.zeros_like(X, dtype=np.float64)
        hx = np.zeros_like(h)
        hy = np.zeros_like(h)
        for a, kx, ky, ph in self.terms:
            arg = kx * X + ky * Y + ph
            h += a * np.sin(arg)
            c = a * np.cos(arg)
            hx += c * kx
            hy += c * ky
        return h, hx, hy


class PanScene:
    """Orthographic top-down camera panning +2 texels per frame over a world
    heightfield; frame t sees world texel (x + 2t, y). Each world texel carries
    a material drawn from the seed: half Lambertian (albedo 0.8), half GGX with
    roughness U(0.05, 1). The G-buffer of frame t is a slice of the world
    arrays, so a texel seen in two frames has bit-identical attributes."""

    def __init__(self, width, height, frames, seed, pan=2, cam_height=100.0,
                 rough_lo=0.05):
        self.W, self.H, self.T, self.pan = width, height, frames, pan
        self.cam_height = cam_height
        ww = width + pan * max(frames, 1)
        X, Y = np.meshgrid(np.arange(ww, dtype=np.float64) + 0.5,
                           np.arange(height, dtype=np.float64) + 0.5)
        h, hx, hy = Heightfield(seed).eval(X, Y)
        n = np.stack([-hx, -hy, np.ones_like(h)], axis=-1)
        n /= np.linalg.norm(n, axis=-1, keepdims=True)
        rng = np.random.default_rng(seed + 7)
        lam = rng.random((height, ww)) < 0.5
        rough = np.where(lam, -1.0, rng.uniform(rough_lo, 1.0, (height, ww)))
        self.world0 = np.concatenate([n, (cam_height - h)[..., None]], -1).astype(np.float32)
        self.world1 = np.stack([np.full_like(h, float(pan)), np.zeros_like(h), rough,
                                np.full_like(h, 0.8)], -1).astype(np.float32)

    def gbuffer(self, t):
        """(g0, g1, g0_prev) of frame t; frame 0 uses its own G-buffer as the
        previous one (the motion vectors still point 2 texels right)."""
        s = self.pan * t
        g0 = np.ascontiguousarray(self.world0[:, s:s + self.W]).reshape(-1, 4)
        g1 = np.ascontiguousarray(self.world1[:, s:s + self.W]).reshape(-1, 4)
        if t == 0:
            return g0, g1, g0
        sp = self.pan * (t - 1)
        g0p = np.ascontiguousarray(self.world0[:, sp:sp + self.W]).reshape(-1, 4)
        return g0, g1, g0p

    def camera(self, t):
        return top_down_camera(x0=float(self.pan * t), y0=0.0, height=self.cam_height)


def masked_lobe_field(seed, n_lobes=4, kappa_lo=5.0, kappa_hi=500.0, constant=0.0):
    rng = np.random.default_rng(seed + 11)
    kap = np.exp(rng.uniform(math.log(kappa_lo), math.log(kappa_hi), n_lobes))
    return Field(dirs=unit_hemisphere_dirs(rng, n_lobes, zmin=0.05), kappas=kap,
                 amps=np.ones(n_lobes), constant=constant, mask=(1.0 / 97.0, 1.0 / 131.0, 0.5))


def workload_pan(width=1920, height=1080, spp=1, frames=60):
    """Plain FP32 guide pass at 1920x1080, 1 spp, 60 frames: camera panning
    2 px/frame over an fBm heightfield with matching motion vectors and depth;
    half the pixels Lambertian, half GGX with roughness U(0.05, 1); radiance =
    4 vMF lobes with kappa log-uniform in [5, 500] times a smooth occlusion
    mask in [0, 1]. The guide starts at mu = (0.5, 0.5), Sigma = 0.1 I, pi = 0.5."""
    seed = SEED_BASE + 2
    sc = PanScene(width, height, frames, seed)
    return dict(params=Params(width, height, spp=spp, seed=seed), camera=sc.camera,
                field=masked_lobe_field(seed), frames=frames, gbuf=sc.gbuffer, scene=sc)


def workload_static(width=1920, height=1080, spp=1, frames=60):
    """The 1080p workload's heightfield, materials and radiance field under a
    static camera (zero motion vectors, the same G-buffer every frame): the
    setting of the temporal-stability measurement, where the difference
    between consecutive images is pure sampling noise."""
    seed = SEED_BASE + 2
    sc = PanScene(width, height, frames, seed, pan=0)
    return dict(params=Params(width, height, spp=spp, seed=seed), camera=sc.camera,
                field=masked_lobe_field(seed), frames=frames, gbuf=sc.gbuffer, scene=sc)


# ----------------------------------------------------------------------------
# Random guide states, directions and sample sets for unit parity.
# ----------------------------------------------------------------------------
def random_gamma(rng, n, k_hi=40, edge_frac=0.1):
    """Guide states as stored moments, exactly representable in float32:
    means anywhere in the square (a share exactly on its edges), spreads
    log-uniform in [0.004, 0.6], correlations in (-0.97, 0.97) (beyond the
    clamp), a share with a negative variance, pi in [0.05, 0.95], k in
    [0, k_hi], I in [0, 3]."""
    mx = rng.uniform(0, 1, n)
    my = rng.uniform(0, 1, n)
    e = rng.random(n) < edge_frac
    mx[e] = rng.choice([0.0, 1.0], e.sum())
    sx = np.exp(rng.uniform(np.log(0.004), np.log(0.6), n))
    sy = np.exp(rng.uniform(np.log(0.004), np.log(0.6), n))
    rho = rng.uniform(-0.97, 0.97, n)
    exx = sx * sx + mx * mx
    eyy = sy * sy + my * my
    exy = rho * sx * sy + mx * my
    neg = rng.random(n) < 0.03
    exx[neg] = mx[neg] * mx[neg] - 1e-3
    g = np.stack([mx, my, exx, eyy, exy, rng.uniform(0.05, 0.95, n),
                  rng.integers(0, k_hi + 1, n).astype(np.float64), rng.uniform(0, 3, n)], 1)
    return g.astype(np.float32)


def random_normals(rng, n, max_tilt=0.6):
    """Unit normals within max_tilt radians of +z (float32, renormalised)."""
    t = rng.uniform(0, max_tilt, n)
    p = rng.uniform(0, 2 * np.pi, n)
    v = np.stack([np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)], 1)
    v = v.astype(np.float32)
    return (v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)


def random_gbuffer(rng, width, height, ggx_frac=0.5, rough_lo=0.02, max_tilt=0.6, glass_frac=0.0):
    """Random normals, depths and materials; a share glass_frac of the pixels
    is transparent (roughness code -2), drawn after the others."""
    hw = width * height
    g0 = np.empty((hw, 4), np.float32)
    g0[:, :3] = random_normals(rng, hw, max_tilt)
    g0[:, 3] = rng.uniform(1.0, 10.0, hw)
    g1 = np.empty((hw, 4), np.float32)
    g1[:, :2] = 0.0
    ggx = rng.random(hw) < ggx_frac
    g1[:, 2] = np.where(ggx, rng.uniform(rough_lo, 1.0, hw), -1.0)
    g1[:, 3] = rng.uniform(0.2, 1.0, hw)
    if glass_frac > 0.0:
        g1[rng.random(hw) < glass_frac, 2] = -2.0
    return g0, g1


def random_directions(rng, n_per_pixel, hw, below_frac=0.05):
    """World directions [n, hw, 3], mostly upper hemisphere of +z, a share below."""
    d = rng.normal(size=(n_per_pixel, hw, 3))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    d[..., 2] = np.abs(d[..., 2])
    flip = rng.random((n_per_pixel, hw)) < below_frac
    d[flip, 2] *= -1.0
    return d.astype(np.float32)


def random_samples(rng, spp, hw):
    """Sample sets for the training step: directions, radiance, estimates and
    strategy bytes (0 BRDF, 1 guide, 2 fallback, +4 wasted draw)."""
    n = spp * hw
    d = random_directions(rng, spp, hw, below_frac=0.02).reshape(n, 3)
    strat = rng.choice(np.array([0, 0, 1, 2], np.uint8), n)
    strat[rng.random(n) < 0.03] |= 4
    return dict(wx=d[:, 0].copy(), wy=d[:, 1].copy(), wz=d[:, 2].copy(),
                radiance=rng.uniform(0.0, 5.0, n).astype(np.float32),
                estimate=rng.uniform(0.0, 3.0, n).astype(np.float32), strategy=strat)


# ----------------------------------------------------------------------------
# Workload 5: 3840x2160 pinhole camera yawing 0.5 deg/frame over a normal-
# mapped ground with 16 occluding quads; GGX everywhere, 8 lobes, 4 spp.
# ----------------------------------------------------------------------------
class _NP:
    """numpy side of the small array interface QuadScene runs on."""
    def __init__(self):
        self.m = np
    def arr(self, x): return np.asarray(x, np.float64)
    def norm(self, x): return np.linalg.norm(x, axis=-1, keepdims=True)
    def cross(self, a, b): return np.cross(a, b)
    def meshgrid(self, a, b): return np.meshgrid(a, b)
    def arange(self, n): return np.arange(n, dtype=np.float64)
    def f32(self, x): return np.asarray(x, np.float32)
    def i64(self, x): return x.astype(np.int64)
    def cat(self, xs): return np.concatenate(xs, -1)


class _TORCH:
    """torch side (on a device) of the same interface, for large screens."""
    def __init__(self, device):
        import torch
        self.m, self.t, self.dev = torch, torch, device
    def arr(self, x): return self.t.as_tensor(np.asarray(x, np.float64), device=self.dev)
    def norm(self, x): return self.t.linalg.norm(x, dim=-1, keepdim=True)
    def cross(self, a, b): return self.t.linalg.cross(a, self.t.broadcast_to(b, a.shape) if b.dim() < a.dim() else b)
    def meshgrid(self, a, b): return self.t.meshgrid(a, b, indexing="xy")
    def arange(self, n): return self.t.arange(n, dtype=self.t.float64, device=self.dev)
    def f32(self, x): return x.to(self.t.float32)
    def i64(self, x): return x.to(self.t.int64)
    def cat(self, xs): return self.t.cat(xs, -1)


class QuadScene:
    """Analytic ray casting of a ground plane z = 0 (normals from a spectral
    fBm, in world units) and n_quads random rectangles above it, seen by a
    pinhole camera that orbits the origin at radius `orbit` and height
    cam_height, looking inward and pitched down, turning yaw_step_deg per
    frame (so nearer quads move against farther ground: parallax and
    disocclusion). Depth is the distance along the primary ray; motion vectors
    come from projecting each hit point into the previous frame's camera.
    Quads are two-sided (normals face the viewer). Roughness is drawn per
    world cell of size 0.25 (GGX U(rough_lo, 1)), albedo 0.8. gbuffer() runs
    in numpy; gbuffer_on(t, device) runs the same arithmetic in torch on a
    device and returns device tensors."""

    def __init__(self, width, height, seed, n_quads=16, hfov_deg=60.0, yaw_step_deg=0.5, pitch_deg=-20.0,
                 cam_height=2.0, orbit=10.0, rough_lo=0.02):
        self.W, self.H = width, height
        self.yaw_step = np.radians(yaw_step_deg)
        self.pitch = np.radians(pitch_deg)
        self.cam_h = cam_height
        self.orbit = orbit
        self.rough_lo = rough_lo
        self.tan_v = np.tan(np.radians(hfov_deg) / 2) * height / width
        self.hf = Heightfield(seed, amplitude=0.05, period=4.0)
        rng = np.random.default_rng(seed + 3)
        # along the arc the camera sweeps in 120 frames, between it and the centre
        ang = rng.uniform(-0.3, 0.3 + np.radians(yaw_step_deg) * 120, n_quads)
        dist = rng.uniform(0.6, 0.9, n_quads) * orbit
        self.qc = np.stack([dist * np.cos(ang), dist * np.sin(ang), rng.uniform(0.3, 1.5, n_quads)], 1)
        e1 = rng.normal(size=(n_quads, 3))
        e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
        e2 = np.cross(e1, rng.normal(size=(n_quads, 3)))
        e2 /= np.linalg.norm(e2, axis=1, keepdims=True)
        self.qe1 = e1 * rng.uniform(0.35, 1.2, (n_quads, 1))
        self.qe2 = e2 * rng.uniform(0.35, 1.2, (n_quads, 1))
        self.rough_seed = seed + 5

    def camera(self, t):
        phi = self.yaw_step * t
        pos = (self.orbit * np.cos(phi), self.orbit * np.sin(phi), self.cam_h)
        yaw = phi + np.pi
        fwd = np.array([np.cos(yaw) * np.cos(self.pitch), np.sin(yaw) * np.cos(self.pitch), np.sin(self.pitch)])
        right = np.cross(fwd, [0.0, 0.0, 1.0])
        right /= np.linalg.norm(right)
        up = np.cross(right, fwd)
        return Camera(1, pos, tuple(fwd), tuple(right), tuple(up), tan_half_fov=float(self.tan_v))

    def _rays(self, X, cam, xs=None, ys=None):
        """Primary rays of every pixel [H, W, 3], or of the pixels (xs, ys) [n, 3]
        (the same arithmetic per pixel)."""
        W, H, m = self.W, self.H, X.m
        if xs is None:
            x = (X.arange(W) + 0.5) / W * 2 - 1
            y = 1 - (X.arange(H) + 0.5) / H * 2
            sx, sy = X.meshgrid(x * self.tan_v * W / H, y * self.tan_v)
        else:
            sx = ((X.arr(xs) + 0.5) / W * 2 - 1) * self.tan_v * W / H
            sy = (1 - (X.arr(ys) + 0.5) / H * 2) * self.tan_v
        f, r, u = X.arr(cam.fwd), X.arr(cam.right), X.arr(cam.up)
        d = f + sx[..., None] * r + sy[..., None] * u
        return d / X.norm(d)

    def _cast(self, X, t, xs=None, ys=None):
        m = X.m
        cam = self.camera(t)
        o = X.arr(cam.origin)
        d = self._rays(X, cam, xs, ys)
        inf = float("inf")
        tg = -o[2] / d[..., 2]
        ground = (d[..., 2] < 0) & (tg > 0)
        tmin = m.where(ground, tg, inf * m.ones_like(tg))
        n = m.zeros_like(d)
        hitq = -1 * m.ones_like(tg)
        for q in range(len(self.qc)):
            e1, e2, c = X.arr(self.qe1[q]), X.arr(self.qe2[q]), X.arr(self.qc[q])
            nq = X.cross(e1[None], e2[None])[0]
            tq = ((c - o) @ nq) / (d @ nq)
            p = o + tq[..., None] * d - c
            a = (p @ e1) / (e1 @ e1)
            b = (p @ e2) / (e2 @ e2)
            hit = (tq > 1e-3) & (tq < tmin) & (m.abs(a) <= 1) & (m.abs(b) <= 1)
            tmin = m.where(hit, tq, tmin)
            hitq = m.where(hit, q + 0.0 * tq, hitq)
            nn = nq / X.norm(nq[None])[0]
            flip = m.where((d @ nn) > 0, -1.0 + 0.0 * tq, 1.0 + 0.0 * tq)
            n = m.where(hit[..., None], nn * flip[..., None], n)
        fin = m.isfinite(tmin)
        P = o + m.where(fin, tmin, 1e3 + 0.0 * tmin)[..., None] * d
        on_ground = (hitq < 0) & fin
        hx, hy = self._slopes(X, P[..., 0], P[..., 1])
        ng = m.stack([-hx, -hy, m.ones_like(hx)], -1)
        ng = ng / X.norm(ng)
        n = m.where(on_ground[..., None], ng, n)
        n = m.where((~fin)[..., None], -d, n)               # no surface: a far wall facing the camera
        depth = m.where(fin, tmin, 1e3 + 0.0 * tmin)
        cell = X.i64(m.floor(P[..., :2] / 0.25))
        h = (cell[..., 0] * 73856093) ^ (cell[..., 1] * 19349663) ^ (X.i64(hitq) + 7) * 83492791 ^ self.rough_seed
        rough = self.rough_lo + (1.0 - self.rough_lo) * ((h & 0xFFFF) / 65535.0)
        return P, n, depth, rough

    def _slopes(self, X, x, y):
        hx, hy = 0.0 * x, 0.0 * x
        for a, kx, ky, ph in self.hf.terms:
            c = a * X.m.cos(kx * x + ky * y + ph)
            hx = hx + c * kx
            hy = hy + c * ky
        return hx, hy

    def _project(self, X, cam, P):
        o, f, r, u = (X.arr(v) for v in (cam.origin, cam.fwd, cam.right, cam.up))
        v = P - o
        cz = v @ f
        sx, sy = (v @ r) / cz, (v @ u) / cz
        px = (sx / (self.tan_v * self.W / self.H) + 1) / 2 * self.W
        py = (1 - sy / self.tan_v) / 2 * self.H
        return px, py, cz

    def _gbuffer(self, X, t):
        m = X.m
        P, n, depth, rough = self._cast(X, t)
        g0 = X.f32(X.cat([n, depth[..., None]])).reshape(-1, 4)
        px, py, cz = self._project(X, self.camera(t - 1), P)
        xs, ys = X.meshgrid(X.arange(self.W) + 0.5, X.arange(self.H) + 0.5)
        mvx = m.where(cz > 0, px - xs, 1e6 + 0.0 * px)
        mvy = m.where(cz > 0, py - ys, 1e6 + 0.0 * py)
        g1 = X.f32(m.stack([mvx, mvy, rough, 0.8 + 0.0 * rough], -1)).reshape(-1, 4)
        if t == 0:
            return g0, g1, g0
        _, n_p, d_p, _ = self._cast(X, t - 1)
        g0p = X.f32(X.cat([n_p, d_p[..., None]])).reshape(-1, 4)
        return g0, g1, g0p

    def surface_at(self, t, xs, ys):
        """(g0, g1) rows of frame t at pixels (xs, ys) only, float32 [n, 4]: the
        same values as the whole frame's G-buffer at those pixels (g1's motion
        vectors are left at zero)."""
        X = _NP()
        _, n, depth, rough = self._cast(X, t, np.asarray(xs, np.float64), np.asarray(ys, np.float64))
        g0 = X.f32(X.cat([n, depth[..., None]]))
        g1 = np.zeros((len(g0), 4), np.float32)
        g1[:, 2] = rough
        g1[:, 3] = 0.8
        return np.ascontiguousarray(g0), g1

    def gbuffer(self, t):
        """(g0, g1, g0_prev) of frame t as float32 numpy arrays."""
        return tuple(np.ascontiguousarray(a) for a in self._gbuffer(_NP(), t))

    def gbuffer_on(self, t, device):
        """(g0, g1, g0_prev) of frame t as contiguous float32 tensors on device."""
        return tuple(a.contiguous() for a in self._gbuffer(_TORCH(device), t))


def coloured(fld, seed):
    """The same field with each lobe and the constant given a colour drawn
    from the seed (channels in [0.2, 1.5] times the monochrome amplitude)."""
    rng = np.random.default_rng(seed + 101)
    n = len(fld.kappas)
    rgb = np.asarray(fld.amps, np.float64)[:, None] * rng.uniform(0.2, 1.5, (n, 3))
    c = tuple(float(fld.constant) * rng.uniform(0.2, 1.5, 3))
    return dataclasses.replace(fld, rgb=rgb, constant_rgb=c)


def eight_lobe_field(seed):
    return masked_lobe_field(seed, n_lobes=8, kappa_lo=5.0, kappa_hi=500.0, constant=0.02)


def workload_4k(width=3840, height=2160, spp=4, frames=120):
    """3840x2160, 4 spp, 120 frames: camera yawing 0.5 deg/frame over a
    normal-mapped ground with 16 random occluding quads (depth discontinuities
    and disocclusions that the depth test rejects); GGX roughness U(0.02, 1)
    everywhere; radiance = 8 vMF lobes x occlusion mask + 0.02. FP16 Gamma, an
    EM step followed by one gradient-refinement step per frame."""
    seed = SEED_BASE + 5
    sc = QuadScene(width, height, seed)
    return dict(params=Params(width, height, spp=spp, seed=seed), camera=sc.camera, field=eight_lobe_field(seed),
                frames=frames, gbuf=sc.gbuffer, scene=sc)
