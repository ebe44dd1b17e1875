"""Context state on the GPU: checkpoint/resume is bit-identical (Philox is
keyed by the frame index, so a resumed run draws the same numbers), a
non-finite Gamma is reported by pg_check, and out-of-order staged calls are
refused without touching Gamma. Failures are made on the host (a NaN
written into Gamma, a call out of order); nothing here faults the device."""
import numpy as np
import pytest

from paper_2112_09728_gb300 import _lib, scenes

from _pg import dev, guide, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_checkpoint_resume_is_bit_identical(dtype):
    import torch
    wl = scenes.workload_pan(128, 48, frames=10)
    par, fld = wl["params"], wl["field"]
    hw = par.width * par.height
    frames = [tuple(dev(a) for a in wl["gbuf"](t)) for t in range(10)]
    a = guide(par, dtype)
    img = torch.empty(hw, device="cuda")
    for t in range(5):
        g0, g1, g0p = frames[t]
        a.pg_frame(g0, g1, wl["camera"](t), g0p, fld, t, img)
    ckpt = a.pg_get_gamma().clone()
    for t in range(5, 10):
        g0, g1, g0p = frames[t]
        a.pg_frame(g0, g1, wl["camera"](t), g0p, fld, t, img)
    end_a, img_a = a.pg_get_gamma().clone(), img.clone()
    b = guide(par, dtype)
    b.pg_set_gamma(dev(host(ckpt)))             # through host memory, as a file would be
    for t in range(5, 10):
        g0, g1, g0p = frames[t]
        b.pg_frame(g0, g1, wl["camera"](t), g0p, fld, t, img)
    assert torch.equal(b.pg_get_gamma(), end_a)
    assert torch.equal(img, img_a)


def test_non_finite_gamma_is_reported_by_pg_check():
    import torch
    W, H = 64, 32
    rng = np.random.default_rng(5)
    g0, g1 = scenes.random_gbuffer(rng, W, H)
    par = scenes.Params(W, H)
    gp = guide(par)
    planes = gp.pg_gamma_to_f32()
    planes[0, 17, 0] = float("nan")             # one pixel's E[X]
    gp.pg_gamma_from_f32(planes)
    img = torch.empty(W * H, device="cuda")
    gp.pg_frame(dev(g0), dev(g1), scenes.top_down_camera(), dev(g0), scenes.two_lobe_field(3), 0, img)
    with pytest.raises(_lib.PgError) as e:
        gp.pg_check()
    assert e.value.status == _lib.PG_ERR_NUMERIC
    gp.pg_check()                               # the flag was cleared by the report


def test_out_of_order_calls_are_refused():
    import torch
    from paper_2112_09728_gb300.guide import alloc_samples
    W, H = 32, 16
    rng = np.random.default_rng(6)
    g0, g1 = scenes.random_gbuffer(rng, W, H)
    par = scenes.Params(W, H)
    gp = guide(par)
    before = gp.pg_get_gamma().clone()
    cam, fld = scenes.top_down_camera(), scenes.two_lobe_field(3)
    s = alloc_samples(1, W * H)
    with pytest.raises(_lib.PgError) as e:
        gp.pg_sample(dev(g0), dev(g1), cam, fld, 0, s)
    assert e.value.status == _lib.PG_ERR_STATE
    with pytest.raises(_lib.PgError) as e:
        gp.pg_update(dev(g0), dev(g1), cam, s)
    assert e.value.status == _lib.PG_ERR_STATE
    gp.pg_reproject(dev(g0), dev(g1), cam, dev(g0))
    with pytest.raises(_lib.PgError) as e:
        gp.pg_frame(dev(g0), dev(g1), cam, dev(g0), fld, 0)
    assert e.value.status == _lib.PG_ERR_STATE
    with pytest.raises(_lib.PgError) as e:
        gp.pg_reproject(dev(g0), dev(g1), cam, dev(g0))
    assert e.value.status == _lib.PG_ERR_STATE
    # the refused calls left Gamma and the staged frame as they were
    gp.pg_sample(dev(g0), dev(g1), cam, fld, 0, s)
    gp.pg_update(dev(g0), dev(g1), cam, s)
    gp.pg_check()
    ref = guide(par)
    ref.pg_set_gamma(before)
    r = alloc_samples(1, W * H)
    ref.pg_reproject(dev(g0), dev(g1), cam, dev(g0))
    ref.pg_sample(dev(g0), dev(g1), cam, fld, 0, r)
    ref.pg_update(dev(g0), dev(g1), cam, r)
    assert torch.equal(gp.pg_get_gamma(), ref.pg_get_gamma())
    # misaligned G-buffer planes are refused on the host
    odd = torch.zeros(W * H * 4 + 1, device="cuda")[1:]
    with pytest.raises((_lib.PgError, ValueError)):
        gp.pg_frame(odd, dev(g1), cam, dev(g0), fld, 0)


@pytest.mark.parametrize("pinned,reuse", [(True, 0), (False, 0), (True, 2)])
def test_frames_from_host_memory_equal_frame_by_frame(pinned, reuse):
    """pg_frames_host (uploads, frames and read-backs overlapped on three
    streams) gives the same Gamma and images, bit for bit, as pg_frame called
    frame by frame on device copies of the same inputs."""
    import dataclasses
    import torch
    n = 7
    wl = scenes.workload_pan(96, 40, frames=n)
    par = dataclasses.replace(wl["params"], reuse_radius=reuse)
    fld, sc = wl["field"], wl["scene"]
    hw = par.width * par.height
    g0h = torch.stack([torch.from_numpy(sc.gbuffer(t)[0]) for t in range(n)]).contiguous()
    g1h = torch.stack([torch.from_numpy(sc.gbuffer(t)[1]) for t in range(n)]).contiguous()
    if pinned:
        g0h, g1h = g0h.pin_memory(), g1h.pin_memory()
    imgh = torch.zeros((n, hw), pin_memory=pinned)
    cams = [sc.camera(t) for t in range(n)]
    a = guide(par, "f16")
    a.pg_frames_host(g0h, g1h, cams, fld, 0, img=imgh)
    b = guide(par, "f16")
    img = torch.empty(hw, device="cuda")
    for t in range(n):
        g0, g1, g0p = (dev(x) for x in sc.gbuffer(t))
        b.pg_frame(g0, g1, cams[t], g0p, fld, t, img)
        assert torch.equal(imgh[t], img.cpu()), t
    assert torch.equal(a.pg_get_gamma(), b.pg_get_gamma())
    # continuing from a given previous g0
    a.pg_frames_host(g0h[n - 1:], g1h[n - 1:], cams[n - 1:], fld, n, g0_prev=g0h[n - 2].contiguous())
    g0, g1, g0p = (dev(x) for x in sc.gbuffer(n - 1))
    b.pg_frame(g0, g1, cams[n - 1], g0p, fld, n)
    assert torch.equal(a.pg_get_gamma(), b.pg_get_gamma())
