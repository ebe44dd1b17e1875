"""Test helpers: build oracle structs and CUDA contexts from the same seeded
inputs (paper_2112_09728_gb300.scenes)."""
import numpy as np

import oracle as O


def ocfg(par, **kw):
    d = dict(width=par.width, height=par.height, spp=par.spp, seed=par.seed, k_max=par.k_max,
             pi_min=par.pi_min, pi_max=par.pi_max, pi_reinit=par.pi_reinit, depth_tol=par.depth_tol,
             normal_tol=par.normal_tol, rough_min=par.rough_min, sigma2_min=par.sigma2_min,
             rho_max=par.rho_max, init_mu=par.init_mu, init_sigma=par.init_sigma,
             reuse_radius=par.reuse_radius, ggx_f0=par.ggx_f0, transparent=par.transparent)
    d.update(kw)
    return O.make_config(**d)


def ocam(cam):
    return O.make_camera(cam.kind, cam.origin, cam.fwd, cam.right, cam.up, cam.pixel_size,
                         cam.tan_half_fov)


def ofld(fld):
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    rgb = getattr(fld, "rgb", None)
    return O.make_field(f32(fld.dirs), f32(fld.kappas), f32(fld.amps),
                        float(np.float32(fld.constant)),
                        None if fld.mask is None else [float(np.float32(m)) for m in fld.mask],
                        None if rgb is None else f32(rgb),
                        None if rgb is None else f32(fld.constant_rgb))


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def guide(par, gamma_dtype="f32", **kw):
    from paper_2112_09728_gb300.guide import GuidePass
    return GuidePass(par.width, par.height, spp=par.spp, gamma_dtype=gamma_dtype, seed=par.seed,
                     k_max=par.k_max, pi_min=par.pi_min, pi_max=par.pi_max, pi_reinit=par.pi_reinit,
                     depth_tol=par.depth_tol, normal_tol=par.normal_tol, rough_min=par.rough_min,
                     sigma2_min=par.sigma2_min, rho_max=par.rho_max, init_mu=par.init_mu,
                     init_sigma=par.init_sigma, init_pi=par.init_pi, reuse_radius=par.reuse_radius,
                     ggx_f0=par.ggx_f0, transparent=par.transparent, **kw)


def set_gamma_rows(gp, rows):
    from paper_2112_09728_gb300.guide import rows_to_planes
    gp.pg_gamma_from_f32(rows_to_planes(dev(np.asarray(rows, np.float32))))


def get_gamma_rows(gp):
    from paper_2112_09728_gb300.guide import planes_to_rows
    return host(planes_to_rows(gp.pg_gamma_to_f32())).astype(np.float64)


def close(a, b, rtol, atol):
    """Elementwise |a - b| <= rtol |b| + atol; returns the worst excess ratio."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    lim = rtol * np.abs(b) + atol
    r = np.abs(a - b) / lim
    return float(r.max()) if r.size else 0.0
