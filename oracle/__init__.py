"""FP64 CPU oracle of the per-pixel guide pass (arXiv 2112.09728).

TEST INFRASTRUCTURE ONLY. The oracle is the plain, slow statement of what the
guide pass computes (pg_oracle.c, double precision, pixel by pixel). Only the
test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package. The product library never imports it, and it never
imports the product package: the two share no code.

Inputs are numpy arrays. G-buffers are float32 ``[H*W, 4]`` planes
(g0 = normal xyz + depth, g1 = motion xy + roughness + albedo). Gamma is float64
``[H*W, 8]`` in the order E[X], E[Y], E[X^2], E[Y^2], E[XY], pi, k, W.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libpg_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile pg_oracle.c with gcc (OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


class Config(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("spp", C.c_int32),
                ("k_max", C.c_int32), ("seed_lo", C.c_uint32), ("seed_hi", C.c_uint32),
                ("pi_min", C.c_double), ("pi_max", C.c_double), ("pi_reinit", C.c_double),
                ("depth_tol", C.c_double), ("normal_tol", C.c_double),
                ("rough_min", C.c_double), ("sigma2_min", C.c_double), ("rho_max", C.c_double),
                ("init_mu", C.c_double * 2), ("init_sigma", C.c_double * 3),
                ("reuse_radius", C.c_int32), ("ggx_f0", C.c_double), ("transparent", C.c_int32)]


class Camera(C.Structure):
    _fields_ = [("kind", C.c_int32), ("origin", C.c_double * 3), ("fwd", C.c_double * 3),
                ("right", C.c_double * 3), ("up", C.c_double * 3),
                ("pixel_size", C.c_double), ("tan_half_fov", C.c_double)]


class Field(C.Structure):
    _fields_ = [("n_lobes", C.c_int32), ("dir", (C.c_double * 3) * 8),
                ("kappa", C.c_double * 8), ("amp", C.c_double * 8), ("constant", C.c_double),
                ("mask_kind", C.c_int32), ("mask", C.c_double * 4), ("rgb", C.c_int32),
                ("amp_rgb", (C.c_double * 3) * 8), ("constant_rgb", C.c_double * 3)]


class Samples(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("wx", "wy", "wz", "radiance", "pdf", "mis", "estimate",
                                           "strategy", "pg", "pb", "ux", "uy", "margin")]


_P = C.c_void_p


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            sig = {
                "or_philox_many": [C.c_int64, _P, _P, _P],
                "or_square_to_hemi": [_P, _P],
                "or_hemi_to_square": [_P, _P],
                "or_basis": [_P, _P, _P],
                "or_gauss_pdf": [_P, _P],
                "or_rect_mass": [_P],
                "or_rect_mass_many": [C.c_int64, _P, _P],
                "or_rect_mass_grad_many": [C.c_int64, _P, _P],
                "or_brdf_cos": [C.c_double, C.c_double, _P, _P],
                "or_brdf_pdf": [C.c_double, _P, _P],
                "or_brdf_sample": [C.c_double, _P, C.c_double, C.c_double, _P, _P],
                "or_radiance": [_P, _P, _P],
                "or_derive_many": [_P, C.c_int64, _P, _P],
                "or_init_gamma": [_P, C.c_double, C.c_int64, _P],
                "or_reproject": [_P, _P, _P, _P, _P, _P, _P, _P],
                "or_sample": [_P, _P, _P, C.c_uint32, _P, _P, _P, _P, _P, _P],
                "or_update": [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
                "or_frame": [_P, _P, _P, C.c_uint32, _P, _P, _P, _P, _P, _P, _P, _P],
                "or_eval": [_P, _P, _P, _P, _P, _P, _P, C.c_int, _P, _P],
                "or_derive_pixels": [_P, _P, _P, _P, _P, _P, _P],
                "or_second_moment": [_P, _P, _P, C.c_uint32, C.c_int, _P, _P, _P, _P, _P, _P, _P],
                "or_adam": [_P, C.c_int64, _P, _P, _P, _P, C.c_double, C.c_double, C.c_double,
                            C.c_double, C.c_double, C.c_double],
                "or_reuse_picks": [_P, C.c_double, C.c_uint32, C.c_uint32, _P, _P, _P],
                "or_frame_pixels": [_P, _P, _P, C.c_uint32, _P, _P, _P, _P, C.c_int64, C.c_int64, _P, _P, _P,
                                    _P, _P, _P],
                "or_brdf_cos_f0": [C.c_double, C.c_double, C.c_double, _P, _P],
                "or_camera_ray": [_P, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P],
                "or_ground_truth": [_P, _P, _P, _P, _P, C.c_int64, _P, _P, C.c_double, _P, _P],
                "or_dielectric_fresnel": [C.c_double],
                "or_set_threads": [C.c_int],
                "or_max_threads": [],
            }
            for name, args in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = None
            lib.or_gauss_pdf.restype = C.c_double
            lib.or_rect_mass.restype = C.c_double
            lib.or_brdf_cos.restype = C.c_double
            lib.or_brdf_pdf.restype = C.c_double
            lib.or_brdf_sample.restype = C.c_int
            lib.or_radiance.restype = C.c_double
            lib.or_reuse_picks.restype = C.c_int
            lib.or_brdf_cos_f0.restype = C.c_double
            lib.or_dielectric_fresnel.restype = C.c_double
            lib.or_max_threads.restype = C.c_int
            _lib = lib
    return _lib


def set_threads(n):
    """Threads of the oracle's parallel loops (for timing; results do not depend on it)."""
    _load().or_set_threads(int(n))


def max_threads():
    return int(_load().or_max_threads())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a if shape is None else a.reshape(shape)


# ----------------------------------------------------------------------------
# structs from plain Python values
# ----------------------------------------------------------------------------
def make_config(width, height, spp=1, seed=0, k_max=32, pi_min=0.05, pi_max=0.95,
                pi_reinit=0.05, depth_tol=0.1, normal_tol=0.9, rough_min=0.1,
                sigma2_min=1e-4, rho_max=0.9, init_mu=(0.5, 0.5),
                init_sigma=(0.1, 0.1, 0.0), reuse_radius=0, ggx_f0=1.0, transparent=0) -> Config:
    """Thresholds that the GPU applies in binary32 are rounded to binary32 here
    so that both sides compare against the same number."""
    f32 = lambda v: float(np.float32(v))
    c = Config()
    c.width, c.height, c.spp, c.k_max = int(width), int(height), int(spp), int(k_max)
    c.seed_lo, c.seed_hi = int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF
    c.pi_min, c.pi_max, c.pi_reinit = f32(pi_min), f32(pi_max), f32(pi_reinit)
    c.depth_tol, c.normal_tol = f32(depth_tol), f32(normal_tol)
    c.rough_min, c.sigma2_min, c.rho_max = f32(rough_min), f32(sigma2_min), f32(rho_max)
    c.init_mu[:] = [f32(v) for v in init_mu]
    c.init_sigma[:] = [f32(v) for v in init_sigma]
    c.reuse_radius = int(reuse_radius)
    c.ggx_f0 = f32(ggx_f0)
    c.transparent = int(transparent)
    return c


def make_camera(kind, origin, fwd, right, up, pixel_size=1.0, tan_half_fov=0.0) -> Camera:
    c = Camera()
    c.kind = int(kind)
    c.origin[:], c.fwd[:], c.right[:], c.up[:] = (list(map(float, v)) for v in
                                                   (origin, fwd, right, up))
    c.pixel_size, c.tan_half_fov = float(pixel_size), float(tan_half_fov)
    return c


def make_field(dirs, kappas, amps, constant=0.0, mask=None, rgb=None, constant_rgb=None) -> Field:
    """rgb: [n, 3] lobe colours (a coloured field; amps then unused)."""
    f = Field()
    n = len(kappas)
    assert n <= 8
    f.n_lobes = n
    for j in range(n):
        f.dir[j][:] = [float(v) for v in dirs[j]]
        f.kappa[j], f.amp[j] = float(kappas[j]), float(amps[j])
    f.constant = float(constant)
    if rgb is not None:
        f.rgb = 1
        for j in range(n):
            f.amp_rgb[j][:] = [float(v) for v in rgb[j]]
        f.constant_rgb[:] = [float(v) for v in (constant_rgb if constant_rgb is not None else (0.0, 0.0, 0.0))]
    if mask is None:
        f.mask_kind = 0
    else:
        f.mask_kind = 1
        f.mask[:] = [float(mask[0]), float(mask[1]), float(mask[2]), 0.0]
    return f


# ----------------------------------------------------------------------------
# elementary functions
# ----------------------------------------------------------------------------
def philox(ctr, key):
    """Philox4x32-10 of each counter row (uint32 [n,4]) under key (uint32 [2])."""
    lib = _load()
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.empty_like(ctr)
    lib.or_philox_many(len(ctr), _ptr(ctr), _ptr(key), _ptr(out))
    return out


def square_to_hemi(u):
    lib = _load()
    u = _f64(u, (-1, 2))
    w = np.empty((len(u), 3))
    for i in range(len(u)):
        lib.or_square_to_hemi(_ptr(u[i]), _ptr(w[i]))
    return w


def hemi_to_square(w):
    lib = _load()
    w = _f64(w, (-1, 3))
    u = np.empty((len(w), 2))
    for i in range(len(w)):
        lib.or_hemi_to_square(_ptr(w[i]), _ptr(u[i]))
    return u


def basis(n):
    lib = _load()
    n = _f64(n, (3,))
    t, b = np.empty(3), np.empty(3)
    lib.or_basis(_ptr(n), _ptr(t), _ptr(b))
    return t, b


def gauss_pdf(g5, u):
    lib = _load()
    return lib.or_gauss_pdf(_ptr(_f64(g5, (5,))), _ptr(_f64(u, (2,))))


def rect_mass(g5):
    """Z for each row of g5 = [mx, my, sxx, syy, sxy]."""
    lib = _load()
    g5 = _f64(g5, (-1, 5))
    z = np.empty(len(g5))
    lib.or_rect_mass_many(len(g5), _ptr(g5), _ptr(z))
    return z


def rect_mass_grad(g5):
    lib = _load()
    g5 = _f64(g5, (-1, 5))
    d = np.empty((len(g5), 5))
    lib.or_rect_mass_grad_many(len(g5), _ptr(g5), _ptr(d))
    return d


def brdf_cos(rough, albedo, wo, wi):
    return _load().or_brdf_cos(float(rough), float(albedo), _ptr(_f64(wo, (3,))),
                               _ptr(_f64(wi, (3,))))


def brdf_cos_f0(rough, albedo, f0, wo, wi):
    return _load().or_brdf_cos_f0(float(rough), float(albedo), float(f0), _ptr(_f64(wo, (3,))),
                                  _ptr(_f64(wi, (3,))))


def dielectric_fresnel(ci):
    return _load().or_dielectric_fresnel(float(ci))


def brdf_pdf(rough, wo, wi):
    return _load().or_brdf_pdf(float(rough), _ptr(_f64(wo, (3,))), _ptr(_f64(wi, (3,))))


def brdf_sample(rough, wo, x1, x2):
    wi = np.empty(3)
    m = C.c_double(0.0)
    ok = _load().or_brdf_sample(float(rough), _ptr(_f64(wo, (3,))), float(x1), float(x2),
                                _ptr(wi), C.byref(m))
    return wi, bool(ok)


def radiance(field, x, w):
    return _load().or_radiance(C.byref(field), _ptr(_f64(x, (3,))), _ptr(_f64(w, (3,))))


def init_gamma(cfg, n, pi=None):
    g = np.empty((n, 8))
    _load().or_init_gamma(C.byref(cfg), float(cfg.pi_reinit if pi is None else pi), n, _ptr(g))
    return g


def derive(cfg, gam):
    gam = _f64(gam, (-1, 8))
    out = np.empty((len(gam), 5))
    _load().or_derive_many(C.byref(cfg), len(gam), _ptr(gam), _ptr(out))
    return out


# ----------------------------------------------------------------------------
# frame-level steps
# ----------------------------------------------------------------------------
def reproject(cfg, g0, g1, g0_prev, gam_prev):
    """Returns (gamma', accept uint8, q int32 (-1 off screen))."""
    hw = cfg.width * cfg.height
    g0, g1, g0p = _f32(g0, (hw, 4)), _f32(g1, (hw, 4)), _f32(g0_prev, (hw, 4))
    gp = _f64(gam_prev, (hw, 8))
    out = np.empty((hw, 8))
    acc = np.empty(hw, np.uint8)
    q = np.empty(hw, np.int32)
    _load().or_reproject(C.byref(cfg), _ptr(g0), _ptr(g1), _ptr(g0p), _ptr(gp), _ptr(out),
                         _ptr(acc), _ptr(q))
    return out, acc, q


_SAMPLE_F64 = ("wx", "wy", "wz", "radiance", "pdf", "mis", "estimate", "pg", "pb", "ux", "uy",
               "margin")


def _alloc_samples(n):
    arrs = {k: np.zeros(n) for k in _SAMPLE_F64}
    arrs["strategy"] = np.zeros(n, np.uint8)
    s = Samples()
    for k, v in arrs.items():
        setattr(s, k, v.ctypes.data)
    return s, arrs


def sample(cfg, cam, field, frame, g0, g1, gam, reinit=None):
    """Sampling step. Returns (samples dict of [spp*HW] arrays, img [HW], or
    [3*HW] planes R, G, B for a coloured field)."""
    hw = cfg.width * cfg.height
    g0, g1 = _f32(g0, (hw, 4)), _f32(g1, (hw, 4))
    gam = _f64(gam, (hw, 8))
    rein = None if reinit is None else np.ascontiguousarray(reinit, np.uint8).reshape(hw)
    s, arrs = _alloc_samples(cfg.spp * hw)
    img = np.empty((3 if field.rgb else 1) * hw)
    _load().or_sample(C.byref(cfg), C.byref(cam), C.byref(field), int(frame) & 0xFFFFFFFF,
                      _ptr(g0), _ptr(g1), _ptr(gam), _ptr(rein), C.byref(s), _ptr(img))
    return arrs, img


def update(cfg, cam, g0, g1, gam, samples, reinit=None):
    """Training step on explicit samples; returns the new gamma."""
    hw = cfg.width * cfg.height
    n = cfg.spp * hw
    g0, g1 = _f32(g0, (hw, 4)), _f32(g1, (hw, 4))
    out = _f64(gam, (hw, 8)).copy()
    rein = None if reinit is None else np.ascontiguousarray(reinit, np.uint8).reshape(hw)
    wx, wy, wz = (_f64(samples[k], (n,)) for k in ("wx", "wy", "wz"))
    rad = _f64(samples["radiance"], (n,))
    strat = np.ascontiguousarray(samples["strategy"], np.uint8).reshape(n)
    _load().or_update(C.byref(cfg), C.byref(cam), _ptr(g0), _ptr(g1), _ptr(out), _ptr(rein),
                      _ptr(wx), _ptr(wy), _ptr(wz), _ptr(rad), _ptr(strat))
    return out


def reuse_picks(cfg, k, pix, frame_idx):
    """Neighbour-VPL picks of one pixel: (dx, dy, sample) int arrays of length N."""
    d = 2 * cfg.reuse_radius + 1
    cmax = max((d * d - 1) * cfg.spp, 1)
    dx, dy, sm = (np.zeros(cmax, np.int32) for _ in range(3))
    n = _load().or_reuse_picks(C.byref(cfg), float(k), int(pix) & 0xFFFFFFFF, int(frame_idx) & 0xFFFFFFFF,
                               _ptr(dx), _ptr(dy), _ptr(sm))
    return dx[:n].copy(), dy[:n].copy(), sm[:n].copy()


def frame_pixels(cfg, cam, field, frame_idx, g0, g1, g0_prev, gam_prev, xs, ys, with_accept=False):
    """Chosen pixels of one frame, each computed alone. gam_prev is either the
    whole previous Gamma [H*W, 8] (gathered at each pixel's reprojected
    pixel) or one row [8] shared by every pixel. Returns (gamma [n, 8], img
    [n] or [n, 3] for a coloured field, margin [n]) and, with with_accept,
    the accept flags [n] as a fourth element."""
    hw = cfg.width * cfg.height
    g0, g1, g0p = _f32(g0, (hw, 4)), _f32(g1, (hw, 4)), _f32(g0_prev, (hw, 4))
    gp = _f64(gam_prev)
    if gp.size == 8:
        gp, stride = gp.reshape(8), 0
    else:
        gp, stride = gp.reshape(hw, 8), 8
    xs = np.ascontiguousarray(xs, np.int32)
    ys = np.ascontiguousarray(ys, np.int32)
    n = len(xs)
    planes = 3 if field.rgb else 1
    out, img, margin = np.empty((n, 8)), np.empty(n * planes), np.empty(n)
    acc = np.empty(n, np.uint8)
    _load().or_frame_pixels(C.byref(cfg), C.byref(cam), C.byref(field), int(frame_idx) & 0xFFFFFFFF,
                            _ptr(g0), _ptr(g1), _ptr(g0p), _ptr(gp), stride, int(n), _ptr(xs), _ptr(ys),
                            _ptr(out), _ptr(img), _ptr(margin), _ptr(acc))
    res = (out, (img if planes == 1 else img.reshape(n, 3)), margin)
    return res + (acc,) if with_accept else res


def frame(cfg, cam, field, frame_idx, g0, g1, g0_prev, gam_prev):
    """One fused frame. Returns (gamma_out, accept, samples dict, img); img is
    [3*HW] (planes R, G, B) for a coloured field."""
    hw = cfg.width * cfg.height
    g0, g1, g0p = _f32(g0, (hw, 4)), _f32(g1, (hw, 4)), _f32(g0_prev, (hw, 4))
    gp = _f64(gam_prev, (hw, 8))
    out = np.empty((hw, 8))
    acc = np.empty(hw, np.uint8)
    s, arrs = _alloc_samples(cfg.spp * hw)
    img = np.empty((3 if field.rgb else 1) * hw)
    _load().or_frame(C.byref(cfg), C.byref(cam), C.byref(field), int(frame_idx) & 0xFFFFFFFF,
                     _ptr(g0), _ptr(g1), _ptr(g0p), _ptr(gp), _ptr(out), _ptr(acc), C.byref(s),
                     _ptr(img))
    return out, acc, arrs, img


def camera_ray(cam, width, height, x, y):
    """Primary ray of pixel (x, y): (origin [3], unit direction [3])."""
    o, d = np.empty(3), np.empty(3)
    _load().or_camera_ray(C.byref(cam), int(width), int(height), int(x), int(y), _ptr(o), _ptr(d))
    return o, d


def ground_truth(cfg, cam, field, g0, g1, xs, ys, tol_rel=1e-8, with_error=False):
    """FP64 ground truth I(p) = int L f_r cos dw of chosen pixels: [n] (or
    [n, 3] for a coloured field); with with_error also the cubature's error
    bound [n]."""
    hw = cfg.width * cfg.height
    g0, g1 = _f32(g0, (hw, 4)), _f32(g1, (hw, 4))
    xs = np.ascontiguousarray(xs, np.int32)
    ys = np.ascontiguousarray(ys, np.int32)
    n = len(xs)
    planes = 3 if field.rgb else 1
    out, err = np.empty(n * planes), np.empty(n)
    _load().or_ground_truth(C.byref(cfg), C.byref(cam), C.byref(field), _ptr(g0), _ptr(g1), int(n), _ptr(xs),
                            _ptr(ys), float(tol_rel), _ptr(out), _ptr(err))
    out = out if planes == 1 else out.reshape(n, 3)
    return (out, err) if with_error else out


EVAL_KEYS = ("pg", "pb", "pmix", "w_guide", "w_brdf", "fcos", "radiance")


def evaluate(cfg, cam, field, g0, g1, gam, dirs, reinit=None):
    """Mixture pieces at caller-given world directions dirs [n, HW, 3]."""
    hw = cfg.width * cfg.height
    dirs = _f64(dirs).reshape(-1, hw, 3)
    n = dirs.shape[0]
    g0, g1 = _f32(g0, (hw, 4)), _f32(g1, (hw, 4))
    gam = _f64(gam, (hw, 8))
    rein = None if reinit is None else np.ascontiguousarray(reinit, np.uint8).reshape(hw)
    out = np.empty((7, n * hw))
    _load().or_eval(C.byref(cfg), C.byref(cam), C.byref(field), _ptr(g0), _ptr(g1), _ptr(gam),
                    _ptr(rein), n, _ptr(np.ascontiguousarray(dirs)), _ptr(out))
    return {k: out[j].reshape(n, hw) for j, k in enumerate(EVAL_KEYS)}


def derive_pixels(cfg, cam, g0, g1, gam, reinit=None):
    """Per pixel: mx, my, sxx, syy, sxy (regularised), Z, pi_eff."""
    hw = cfg.width * cfg.height
    g0, g1 = _f32(g0, (hw, 4)), _f32(g1, (hw, 4))
    gam = _f64(gam, (hw, 8))
    rein = None if reinit is None else np.ascontiguousarray(reinit, np.uint8).reshape(hw)
    out = np.empty((hw, 8))
    _load().or_derive_pixels(C.byref(cfg), C.byref(cam), _ptr(g0), _ptr(g1), _ptr(gam),
                             _ptr(rein), _ptr(out))
    return out[:, :7]


def theta_from_gamma(cfg, gam):
    """Regularised (mu_x, mu_y, s_xx, s_yy, s_xy) and the stored pi: [HW, 6]."""
    gam = _f64(gam, (-1, 8))
    return np.concatenate([derive(cfg, gam), gam[:, 5:6]], 1)


def second_moment(cfg, cam, field, frame, n, g0, g1, theta0, theta=None):
    """Loss [HW], gradient [HW, 6] and smallest decision margin [HW] of the
    second-moment loss with n draws per pixel from theta0 held fixed."""
    hw = cfg.width * cfg.height
    g0, g1 = _f32(g0, (hw, 4)), _f32(g1, (hw, 4))
    t0 = _f64(theta0, (hw, 6))
    t = None if theta is None else _f64(theta, (hw, 6))
    loss, grad, margin = np.empty(hw), np.empty((hw, 6)), np.empty(hw)
    _load().or_second_moment(C.byref(cfg), C.byref(cam), C.byref(field), int(frame) & 0xFFFFFFFF, int(n),
                             _ptr(g0), _ptr(g1), _ptr(t0), _ptr(t), _ptr(loss), _ptr(grad), _ptr(margin))
    return loss, grad, margin


def adam(cfg, gam, grad, m, v, lr, b1, b2, eps, step):
    """One projected Adam step on theta; returns (gamma, m, v)."""
    gam = _f64(gam, (-1, 8)).copy()
    n = len(gam)
    grad = _f64(grad, (n, 6))
    m, v = _f64(m, (n, 6)).copy(), _f64(v, (n, 6)).copy()
    c1, c2 = 1.0 / (1.0 - b1 ** step), 1.0 / (1.0 - b2 ** step)
    _load().or_adam(C.byref(cfg), n, _ptr(gam), _ptr(grad), _ptr(m), _ptr(v), float(lr), float(b1),
                    float(b2), float(eps), c1, c2)
    return gam, m, v
