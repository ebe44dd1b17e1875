"""pg_frame_noalloc: a whole staged frame for callers that cannot allocate
device memory (an engine that hands out all device memory through its own
allocator, code that must not allocate while frames are in flight). Its only
scratch, the work copy of Gamma, lives in a fixed array inside the library.

Checked here: two consecutive frames through the entry point agree with the
same frames through the context's staged calls (pg_reproject, pg_sample,
pg_update), within the tolerance of the other parity tests; the second call
leaves the device's free memory unchanged; and a screen larger than the fixed
scratch is refused.
"""
import numpy as np
import pytest

from paper_2112_09728_gb300 import scenes

from _pg import close, dev, guide, host

pytestmark = pytest.mark.gpu


def _as_float(raw, dtype):
    import torch
    a = host(raw)
    if dtype == "f32":
        return a.view(np.float32).astype(np.float64)
    if dtype == "f16":
        return a.view(np.float16).astype(np.float64)
    return torch.from_numpy(a.copy()).view(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("dtype,sr,in_place", [("f32", 0, False), ("f16", 0, False), ("bf16", 0, False),
                                               ("f16", 1, False), ("bf16", 1, False), ("f16", 0, True)])
def test_frame_noalloc_matches_the_staged_entry_points(dtype, sr, in_place):
    """Two frames in a row through pg_frame_noalloc against the same frames
    through a context's staged calls: storage forms FP32, FP16 and BF16, with
    stochastic rounding of the 16-bit store, and in place (Gamma in = out)."""
    import torch
    from paper_2112_09728_gb300.guide import alloc_samples, pg_frame_noalloc

    wl = scenes.workload_pan(96, 40, frames=3)
    par, fld = wl["params"], wl["field"]
    hw = par.width * par.height
    gp = guide(par, dtype, stochastic_round=sr)
    g_in = gp.pg_get_gamma().clone()          # the initial Gamma written by pg_create
    g_out = g_in if in_place else torch.empty_like(g_in)
    sa, sb = alloc_samples(par.spp, hw), alloc_samples(par.spp, hw)
    ia, ib = torch.empty(hw, device="cuda"), torch.empty(hw, device="cuda")
    frames = [tuple(dev(a) for a in wl["gbuf"](t)) for t in range(2)]
    torch.cuda.synchronize()
    free_after_first = None
    for t in range(2):
        g0, g1, g0p = frames[t]
        cam = wl["camera"](t)
        gp.pg_reproject(g0, g1, cam, g0p)
        gp.pg_sample(g0, g1, cam, fld, t, sa, ia)
        gp.pg_update(g0, g1, cam, sa)
        ref = gp.pg_get_gamma()
        pg_frame_noalloc(gp.cfg, g0, g1, cam, g0p, fld, t, g_in, g_out, sb, ib)
        torch.cuda.synchronize()
        if t == 0:
            free_after_first = torch.cuda.mem_get_info()[0]
        else:
            assert torch.cuda.mem_get_info()[0] == free_after_first
        # the same kernels on the same inputs: bit-identical Gamma
        assert np.array_equal(host(g_out), host(ref))
        assert close(_as_float(g_out, dtype), _as_float(ref, dtype), 1e-5, 1e-6) <= 1.0
        assert close(host(ib), host(ia), 1e-5, 1e-6) <= 1.0
        for k in ("wx", "wy", "wz", "radiance", "pdf", "mis", "estimate"):
            assert close(host(sb[k]), host(sa[k]), 1e-5, 1e-6) <= 1.0
        assert (host(sb["strategy"]) == host(sa["strategy"])).all()
        if not in_place:
            g_in, g_out = g_out, g_in
    gp.close()


def test_frame_noalloc_refuses_screens_beyond_its_scratch():
    import torch
    from paper_2112_09728_gb300 import _lib
    from paper_2112_09728_gb300.guide import alloc_samples, make_config, pg_frame_noalloc

    W, H = 640, 480   # 307,200 pixels > 262,144
    cfg = make_config(W, H)
    g = torch.zeros(W * H * 4, device="cuda")
    gam = torch.zeros(W * H * 32, dtype=torch.uint8, device="cuda")
    s = alloc_samples(1, W * H)
    with pytest.raises(_lib.PgError) as e:
        pg_frame_noalloc(cfg, g, g, scenes.top_down_camera(), g, scenes.two_lobe_field(1), 0, gam, gam, s)
    assert e.value.status == _lib.PG_ERR_ARG
