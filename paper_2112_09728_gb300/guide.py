"""Thin torch-facing binding of the guide-pass C ABI (include/pg.h).

Argument marshalling only: every step of the pass runs in libpg.so. Tensors
must be CUDA, contiguous and of the documented dtype; calls are enqueued on
torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L

_DTYPES = {"f32": L.PG_F32, "f16": L.PG_F16, "bf16": L.PG_BF16}
SAMPLE_FLOAT_PLANES = ("wx", "wy", "wz", "radiance", "pdf", "mis", "estimate")
EVAL_KEYS = ("pg", "pb", "pmix", "w_guide", "w_brdf", "fcos", "radiance")


def _ptr(t, dtype=torch.float32, what="tensor", align16=False):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % what)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (what, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    p = t.data_ptr()
    if align16 and p % 16:
        raise ValueError("%s must be 16-byte aligned" % what)
    return p


def make_camera(cam) -> L.pg_camera:
    c = L.pg_camera()
    c.kind = int(cam.kind)
    for name in ("origin", "fwd", "right", "up"):
        getattr(c, name)[:] = [float(v) for v in getattr(cam, name)]
    c.pixel_size = float(cam.pixel_size)
    c.tan_half_fov = float(cam.tan_half_fov)
    return c


def make_field(fld) -> L.pg_field:
    f = L.pg_field()
    n = len(fld.kappas)
    if n > 8:
        raise ValueError("at most 8 lobes")
    f.n_lobes = n
    for j in range(n):
        f.dir[j][:] = [float(v) for v in fld.dirs[j]]
        f.kappa[j] = float(fld.kappas[j])
        f.amp[j] = float(fld.amps[j])
    f.constant = float(fld.constant)
    if getattr(fld, "rgb", None) is not None:
        f.rgb = 1
        for j in range(n):
            f.amp_rgb[j][:] = [float(v) for v in fld.rgb[j]]
        f.constant_rgb[:] = [float(v) for v in (fld.constant_rgb or (0.0, 0.0, 0.0))]
    if fld.mask is None:
        f.mask_kind = 0
    else:
        f.mask_kind = 1
        f.mask[:] = [float(fld.mask[0]), float(fld.mask[1]), float(fld.mask[2]), 0.0]
    return f


def alloc_samples(spp, hw, device="cuda"):
    d = {k: torch.empty(spp * hw, dtype=torch.float32, device=device) for k in SAMPLE_FLOAT_PLANES}
    d["strategy"] = torch.empty(spp * hw, dtype=torch.uint8, device=device)
    return d


def make_config(width, height, spp=1, gamma_dtype="f32", seed=0, **overrides) -> L.pg_config:
    """pg_config with the library's defaults and the given overrides."""
    cfg = L.pg_config()
    L.load(overrides.pop("bounds_check", False)).pg_config_default(C.byref(cfg), int(width), int(height))
    cfg.spp = int(spp)
    cfg.gamma_dtype = _DTYPES[gamma_dtype]
    cfg.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    for k, v in overrides.items():
        if k in ("init_mu", "init_sigma"):
            getattr(cfg, k)[:] = [float(x) for x in v]
        elif k in ("k_max", "reuse_radius", "stochastic_round", "transparent"):
            setattr(cfg, k, int(v))
        elif k == "adam_dtype":
            cfg.adam_dtype = _DTYPES[v] if isinstance(v, str) else int(v)
        else:
            setattr(cfg, k, float(v))
    return cfg


class GuidePass:
    """One guide-pass context (pg_ctx): owns Gamma on the current device."""

    def __init__(self, width, height, spp=1, gamma_dtype="f32", seed=0, bounds_check=False, **overrides):
        """bounds_check: run on the bounds-checked build of the library
        (libpg_bounds.so), whose pg_check reports PG_ERR_BOUNDS for an index
        outside its buffer."""
        self._lib = L.load(bounds_check)
        cfg = make_config(width, height, spp, gamma_dtype, seed, bounds_check=bounds_check, **overrides)
        self.cfg = cfg
        self.width, self.height, self.spp = int(width), int(height), int(spp)
        self.hw = self.width * self.height
        self.gamma_dtype = gamma_dtype
        h = C.c_void_p()
        st = self._lib.pg_create(C.byref(cfg), C.c_void_p(self._stream()), C.byref(h))
        if st != L.PG_OK or not h.value:
            raise L.PgError(st, "pg_create")
        self._h = h

    # -- plumbing ---------------------------------------------------------
    @staticmethod
    def _stream():
        return torch.cuda.current_stream().cuda_stream

    def _call(self, name, *args):
        self._lib.pg_set_stream(self._h, C.c_void_p(self._stream()))
        st = getattr(self._lib, name)(self._h, *args)
        if st != L.PG_OK:
            msg = self._lib.pg_last_error(self._h)
            raise L.PgError(st, name, msg.decode() if msg else "")

    def _gbuf(self, g0, g1, camera):
        gb = L.pg_gbuffer()
        gb.g0 = _ptr(g0, what="g0", align16=True)
        gb.g1 = _ptr(g1, what="g1", align16=True)
        self._check_len(g0, 4 * self.hw, "g0")
        self._check_len(g1, 4 * self.hw, "g1")
        gb.camera = make_camera(camera)
        return gb

    @staticmethod
    def _check_len(t, n, what):
        if t.numel() != n:
            raise ValueError("%s must have %d elements, has %d" % (what, n, t.numel()))

    def _samples(self, s, required=()):
        ps = L.pg_samples()
        n = self.spp * self.hw
        for k in SAMPLE_FLOAT_PLANES:
            t = None if s is None else s.get(k)
            if t is not None:
                self._check_len(t, n, k)
            setattr(ps, k, _ptr(t, what=k))
        t = None if s is None else s.get("strategy")
        if t is not None:
            self._check_len(t, n, "strategy")
        ps.strategy = _ptr(t, dtype=torch.uint8, what="strategy")
        return ps

    # -- the C ABI, one method per entry point ----------------------------
    def pg_reproject(self, g0, g1, camera, g0_prev, accept=None):
        self._check_len(g0_prev, 4 * self.hw, "g0_prev")
        if accept is not None:
            self._check_len(accept, self.hw, "accept")
        self._call("pg_reproject", C.byref(self._gbuf(g0, g1, camera)),
                   C.c_void_p(_ptr(g0_prev, what="g0_prev", align16=True)),
                   C.c_void_p(_ptr(accept, dtype=torch.uint8, what="accept")))

    @staticmethod
    def image_planes(field):
        """1, or 3 for a coloured field (R, G, B planes)."""
        return 3 if getattr(field, "rgb", None) is not None else 1

    def pg_sample(self, g0, g1, camera, field, frame, samples=None, img=None):
        if img is not None:
            self._check_len(img, self.image_planes(field) * self.hw, "img")
        ps = self._samples(samples)
        self._call("pg_sample", C.byref(self._gbuf(g0, g1, camera)), C.byref(make_field(field)),
                   C.c_uint32(int(frame) & 0xFFFFFFFF), C.byref(ps), C.c_void_p(_ptr(img, what="img")))

    def pg_update(self, g0, g1, camera, samples):
        self._call("pg_update", C.byref(self._gbuf(g0, g1, camera)), C.byref(self._samples(samples)))

    def pg_frame(self, g0, g1, camera, g0_prev, field, frame, img=None):
        self._check_len(g0_prev, 4 * self.hw, "g0_prev")
        if img is not None:
            self._check_len(img, self.image_planes(field) * self.hw, "img")
        self._call("pg_frame", C.byref(self._gbuf(g0, g1, camera)),
                   C.c_void_p(_ptr(g0_prev, what="g0_prev", align16=True)), C.byref(make_field(field)),
                   C.c_uint32(int(frame) & 0xFFFFFFFF), C.c_void_p(_ptr(img, what="img")))

    def pg_frames_host(self, g0, g1, cameras, field, frame0, g0_prev=None, img=None):
        """n whole frames from host memory: g0, g1 CPU float32 tensors [n, H*W, 4]
        (page-locked for overlapped copies), cameras a list of n cameras,
        g0_prev the g0 before frame 0 (CPU [H*W, 4] or None), img a CPU float32
        tensor [n, planes * H*W] for the estimates (planes = 3 for a coloured
        field) or None. Returns img."""
        n = len(cameras)
        for t, what in ((g0, "g0"), (g1, "g1")):
            if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
                raise TypeError("%s must be a contiguous float32 CPU tensor" % what)
            self._check_len(t, n * 4 * self.hw, what)
        if g0_prev is not None:
            if g0_prev.is_cuda or g0_prev.dtype != torch.float32 or not g0_prev.is_contiguous():
                raise TypeError("g0_prev must be a contiguous float32 CPU tensor")
            self._check_len(g0_prev, 4 * self.hw, "g0_prev")
        if img is not None:
            if img.is_cuda or img.dtype != torch.float32 or not img.is_contiguous():
                raise TypeError("img must be a contiguous float32 CPU tensor")
            self._check_len(img, n * self.image_planes(field) * self.hw, "img")
        cams = (L.pg_camera * n)(*[make_camera(c) for c in cameras])
        self._call("pg_frames_host", C.c_int32(n), C.c_void_p(g0.data_ptr()), C.c_void_p(g1.data_ptr()), cams,
                   C.byref(make_field(field)), C.c_uint32(int(frame0) & 0xFFFFFFFF),
                   C.c_void_p(None if g0_prev is None else g0_prev.data_ptr()),
                   C.c_void_p(None if img is None else img.data_ptr()))
        return img

    def pg_eval(self, g0, g1, camera, field, dirs, out=None):
        """dirs [n, H*W, 3] float32 -> dict of [n, H*W] planes (EVAL_KEYS)."""
        n = dirs.numel() // (3 * self.hw)
        self._check_len(dirs, 3 * n * self.hw, "dirs")
        if out is None:
            out = torch.empty(7 * n * self.hw, dtype=torch.float32, device=dirs.device)
        self._call("pg_eval", C.byref(self._gbuf(g0, g1, camera)), C.byref(make_field(field)), C.c_int32(n),
                   C.c_void_p(_ptr(dirs, what="dirs")), C.c_void_p(_ptr(out, what="out")))
        o = out.view(7, n, self.hw)
        return {k: o[j] for j, k in enumerate(EVAL_KEYS)}

    def pg_grad(self, g0, g1, camera, field, frame, n_samples, theta=None, loss=None, grad=None):
        """Second-moment loss [H*W] and its gradient [6, H*W] at theta (default:
        the current Gamma's), n_samples draws per pixel."""
        if theta is not None:
            self._check_len(theta, 6 * self.hw, "theta")
        if loss is None:
            loss = torch.empty(self.hw, dtype=torch.float32, device="cuda")
        if grad is None:
            grad = torch.empty((6, self.hw), dtype=torch.float32, device="cuda")
        self._call("pg_grad", C.byref(self._gbuf(g0, g1, camera)), C.byref(make_field(field)),
                   C.c_uint32(int(frame) & 0xFFFFFFFF), C.c_int32(int(n_samples)),
                   C.c_void_p(_ptr(theta, what="theta")), C.c_void_p(_ptr(loss, what="loss")),
                   C.c_void_p(_ptr(grad, what="grad")))
        return loss, grad

    def pg_adam_step(self, grad, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8, step=1):
        self._check_len(grad, 6 * self.hw, "grad")
        self._call("pg_adam_step", C.c_void_p(_ptr(grad, what="grad")), C.c_float(lr), C.c_float(beta1),
                   C.c_float(beta2), C.c_float(eps), C.c_int32(int(step)))

    def pg_get_adam_state(self, m=None, v=None):
        """The Adam moments (m, v) as float32 [6, H*W] planes."""
        if m is None:
            m = torch.empty((6, self.hw), dtype=torch.float32, device="cuda")
        if v is None:
            v = torch.empty((6, self.hw), dtype=torch.float32, device="cuda")
        self._check_len(m, 6 * self.hw, "m")
        self._check_len(v, 6 * self.hw, "v")
        self._call("pg_get_adam_state", C.c_void_p(_ptr(m, what="m")), C.c_void_p(_ptr(v, what="v")))
        return m, v

    def pg_set_adam_state(self, m, v):
        self._check_len(m, 6 * self.hw, "m")
        self._check_len(v, 6 * self.hw, "v")
        self._call("pg_set_adam_state", C.c_void_p(_ptr(m, what="m")), C.c_void_p(_ptr(v, what="v")))

    def pg_theta_from_gamma(self, theta=None):
        if theta is None:
            theta = torch.empty((6, self.hw), dtype=torch.float32, device="cuda")
        self._call("pg_theta_from_gamma", C.c_void_p(_ptr(theta, what="theta")))
        return theta

    def pg_theta_to_gamma(self, theta):
        self._check_len(theta, 6 * self.hw, "theta")
        self._call("pg_theta_to_gamma", C.c_void_p(_ptr(theta, what="theta")))

    def gamma_bytes(self):
        return int(self._lib.pg_gamma_bytes(self._h))

    def pg_get_gamma(self, dst=None):
        """Raw Gamma bytes (uint8 CUDA tensor) in the storage layout."""
        if dst is None:
            dst = torch.empty(self.gamma_bytes(), dtype=torch.uint8, device="cuda")
        self._call("pg_get_gamma", C.c_void_p(_ptr(dst, dtype=torch.uint8, what="dst")), C.c_int32(0))
        return dst

    def pg_set_gamma(self, src):
        self._check_len(src, self.gamma_bytes(), "src")
        self._call("pg_set_gamma", C.c_void_p(_ptr(src, dtype=torch.uint8, what="src")), C.c_int32(0))

    def pg_gamma_to_f32(self, dst=None):
        """Gamma as float32 [2, H*W, 4] raw-moment planes."""
        if dst is None:
            dst = torch.empty((2, self.hw, 4), dtype=torch.float32, device="cuda")
        self._call("pg_gamma_to_f32", C.c_void_p(_ptr(dst, what="dst", align16=True)))
        return dst

    def pg_gamma_from_f32(self, src):
        self._check_len(src, 8 * self.hw, "src")
        self._call("pg_gamma_from_f32", C.c_void_p(_ptr(src, what="src", align16=True)))

    def pg_get_reprojected(self, dst=None):
        if dst is None:
            dst = torch.empty((2, self.hw, 4), dtype=torch.float32, device="cuda")
        self._call("pg_get_reprojected", C.c_void_p(_ptr(dst, what="dst", align16=True)))
        return dst

    def pg_check(self):
        self._call("pg_check")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.pg_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pg_philox(ctr, key, use_curand=False):
    """Philox4x32-10 of each row of ctr (uint32-valued int32 CUDA tensor [n, 4])."""
    lib = L.load()
    out = torch.empty_like(ctr)
    k = (C.c_uint32 * 2)(int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF)
    st = lib.pg_philox(C.c_void_p(_ptr(ctr, dtype=torch.int32, what="ctr", align16=True)), k,
                       C.c_int64(ctr.shape[0]), C.c_void_p(_ptr(out, dtype=torch.int32, what="out", align16=True)),
                       C.c_int32(1 if use_curand else 0), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != L.PG_OK:
        raise L.PgError(st, "pg_philox")
    return out


def pg_frame_noalloc(cfg, g0, g1, camera, g0_prev, field, frame, gamma_in, gamma_out, samples, img=None):
    """One staged frame without a context and without device allocation (see
    include/pg.h). gamma_in / gamma_out: uint8 CUDA tensors of the storage
    layout's size (H*W*32 bytes for f32, H*W*16 for f16/bf16; the same tensor
    for an in-place frame); samples: dict of sample planes (alloc_samples:
    spp*H*W elements each; wx, wy, wz, radiance and strategy required); img:
    the per-pixel estimate (H*W, or 3*H*W planes for a coloured field) or
    None. Every size is checked here: the C entry point cannot see the
    tensors' sizes, and a short buffer would be read and written out of
    bounds on the device."""
    lib = L.load()
    hw = int(cfg.width) * int(cfg.height)
    n = int(cfg.spp) * hw
    gbytes = hw * (32 if int(cfg.gamma_dtype) == L.PG_F32 else 16)
    checks = [(g0, 4 * hw, "g0"), (g1, 4 * hw, "g1"), (g0_prev, 4 * hw, "g0_prev"),
              (gamma_in, gbytes, "gamma_in"), (gamma_out, gbytes, "gamma_out")]
    for k in ("wx", "wy", "wz", "radiance", "strategy"):
        if samples.get(k) is None:
            raise ValueError("samples[%r] is required" % k)
    checks += [(samples[k], n, "samples[%r]" % k) for k in SAMPLE_FLOAT_PLANES + ("strategy",)
               if samples.get(k) is not None]
    if img is not None:
        checks.append((img, GuidePass.image_planes(field) * hw, "img"))
    for t, want, what in checks:
        if not isinstance(t, torch.Tensor):
            raise TypeError("%s must be a tensor" % what)
        if t.numel() != want:
            raise ValueError("%s must have %d elements, has %d" % (what, want, t.numel()))
    gb = L.pg_gbuffer()
    gb.g0 = _ptr(g0, what="g0", align16=True)
    gb.g1 = _ptr(g1, what="g1", align16=True)
    gb.camera = make_camera(camera)
    ps = L.pg_samples()
    for k in SAMPLE_FLOAT_PLANES:
        setattr(ps, k, _ptr(samples.get(k), what=k))
    ps.strategy = _ptr(samples.get("strategy"), dtype=torch.uint8, what="strategy")
    st = lib.pg_frame_noalloc(C.byref(cfg), C.byref(gb), C.c_void_p(_ptr(g0_prev, what="g0_prev", align16=True)),
                              C.byref(make_field(field)), C.c_uint32(int(frame) & 0xFFFFFFFF),
                              C.c_void_p(_ptr(gamma_in, dtype=torch.uint8, what="gamma_in", align16=True)),
                              C.c_void_p(_ptr(gamma_out, dtype=torch.uint8, what="gamma_out", align16=True)),
                              C.byref(ps), C.c_void_p(_ptr(img, what="img")),
                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != L.PG_OK:
        raise L.PgError(st, "pg_frame_noalloc")


def planes_to_rows(planes):
    """[2, HW, 4] raw-moment planes -> [HW, 8] rows (E[X], E[Y], E[X^2], E[Y^2], E[XY], pi, k, W)."""
    return torch.cat([planes[0], planes[1]], dim=1)


def rows_to_planes(rows):
    return torch.stack([rows[:, :4], rows[:, 4:]], 0).contiguous()


class PgSecondMoment(torch.autograd.Function):
    """Per-pixel Monte Carlo second moment of the guided estimator as a
    function of theta [6, H*W]; forward and backward both come from pg_grad's
    kernel (the draws are held fixed, so the gradient is exact for them)."""

    @staticmethod
    def forward(ctx, theta, guide, g0, g1, camera, field, frame, n_samples):
        loss, grad = guide.pg_grad(g0, g1, camera, field, frame, n_samples, theta=theta.detach().contiguous())
        ctx.save_for_backward(grad)
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        (grad,) = ctx.saved_tensors
        return grad_loss[None, :] * grad, None, None, None, None, None, None, None
