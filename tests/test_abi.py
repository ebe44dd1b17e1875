"""The C-ABI library builds, loads and exports every symbol include/*.h
declares; host-side argument checks need no GPU."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(pg_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2112_09728_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    d = _declared()
    for n in ("pg_create", "pg_reproject", "pg_sample", "pg_update", "pg_frame", "pg_destroy"):
        assert n in d


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2112_09728_gb300 import _lib
    checked = _lib.load(bounds_check=True)          # the bounds-checked build exports the same ABI
    missing = [n for n in sorted(_declared()) if not hasattr(checked, n)]
    assert not missing, missing


def test_reuse_pick_decode_is_exact_in_binary32():
    """The training pass decodes candidate o of the (2R+1)^2 - 1 window cells
    x spp samples with binary32 floor divisions, cell = floor((o + 0.5) *
    fl(1/spp)) and row = floor((cell + 0.5) * fl(1/(2R+1))), to avoid integer
    division. Both equal the integer quotients for every candidate of every
    configuration the library accepts (spp <= 1024, R <= 8)."""
    import numpy as np
    f32 = np.float32
    for spp in range(2, 1025):
        c = (17 * 17 - 1) * spp                     # the largest window; smaller ones are prefixes
        o = np.arange(c, dtype=np.int64)
        inv = f32(1) / f32(spp)
        cell = ((o.astype(f32) + f32(0.5)) * inv).astype(np.int64)     # truncation of a positive value
        assert np.array_equal(cell, o // spp), spp
    for r in range(1, 9):
        d = 2 * r + 1
        cell = np.arange(d * d, dtype=np.int64)
        row = ((cell.astype(f32) + f32(0.5)) * (f32(1) / f32(d))).astype(np.int64)
        assert np.array_equal(row, cell // d), r


def test_binding_covers_every_declared_symbol(lib):
    from paper_2112_09728_gb300 import _lib
    assert _declared() <= set(_lib.exported_names())


def test_ctypes_mirror_of_pg_config_follows_the_header():
    """The binding's pg_config has the header's fields, in the header's
    order, so every field lands where the library reads it."""
    from paper_2112_09728_gb300 import _lib
    src = open(os.path.join(ROOT, "include", "pg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\} pg_config;", src).group(1)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(None, 1)[1].split(","):
            names.append(re.sub(r"\[.*\]", "", part).strip())
    assert names == [f[0] for f in _lib.pg_config._fields_]


def test_config_default_and_validation_without_gpu(lib):
    from paper_2112_09728_gb300 import _lib
    cfg = _lib.pg_config()
    lib.pg_config_default(C.byref(cfg), 1920, 1080)
    assert (cfg.width, cfg.height, cfg.spp, cfg.k_max) == (1920, 1080, 1, 32)
    assert abs(cfg.pi_min - 0.05) < 1e-7 and abs(cfg.pi_max - 0.95) < 1e-7
    assert abs(cfg.pi_reinit - 0.05) < 1e-7
    h = C.c_void_p()
    # invalid configurations are rejected on the host before any device work
    for field, bad in (("width", 0), ("height", 32769), ("spp", 0), ("spp", 1025), ("gamma_dtype", 7),
                       ("pi_min", 0.99), ("rho_max", 1.0), ("sigma2_min", 0.0), ("reuse_radius", 9),
                       ("reuse_radius", -1), ("stochastic_round", 2), ("ggx_f0", 1.5), ("ggx_f0", -0.1),
                       ("transparent", 2), ("adam_dtype", 1), ("adam_dtype", 3)):
        c2 = _lib.pg_config()
        C.memmove(C.byref(c2), C.byref(cfg), C.sizeof(cfg))
        setattr(c2, field, bad)
        assert lib.pg_create(C.byref(c2), None, C.byref(h)) == _lib.PG_ERR_ARG
        assert not h.value
    assert lib.pg_create(None, None, C.byref(h)) == _lib.PG_ERR_ARG
    # NULL contexts are rejected, not dereferenced
    assert lib.pg_frame(None, None, None, None, 0, None) == _lib.PG_ERR_ARG
    assert lib.pg_reproject(None, None, None, None) == _lib.PG_ERR_ARG
    assert lib.pg_frames_host(None, 1, None, None, None, None, 0, None, None) == _lib.PG_ERR_ARG
    assert lib.pg_check(None) == _lib.PG_ERR_ARG
    assert lib.pg_get_adam_state(None, None, None) == _lib.PG_ERR_ARG
    assert lib.pg_set_adam_state(None, None, None) == _lib.PG_ERR_ARG
    assert lib.pg_gamma_bytes(None) == 0
    lib.pg_destroy(None)


def test_frame_noalloc_binding_checks_every_size_before_the_call():
    """The C entry point cannot see buffer sizes: the binding refuses a short
    Gamma, sample plane or image with ValueError before anything reaches the
    library (CPU tensors suffice, no call is made)."""
    import torch
    from paper_2112_09728_gb300 import scenes
    from paper_2112_09728_gb300.guide import alloc_samples, make_config, pg_frame_noalloc

    W, H = 8, 4
    hw = W * H
    cfg = make_config(W, H, spp=2, gamma_dtype="f16")
    g = torch.zeros(4 * hw)
    cam, fld = scenes.top_down_camera(), scenes.two_lobe_field(1)
    ok = dict(g0=g, g1=g, g0_prev=g, gamma_in=torch.zeros(16 * hw, dtype=torch.uint8),
              gamma_out=torch.zeros(16 * hw, dtype=torch.uint8), samples=alloc_samples(2, hw, device="cpu"),
              img=torch.zeros(hw))

    def call(**kw):
        a = dict(ok, **kw)
        pg_frame_noalloc(cfg, a["g0"], a["g1"], cam, a["g0_prev"], fld, 0, a["gamma_in"], a["gamma_out"],
                         a["samples"], a["img"])

    bad = [dict(gamma_in=torch.zeros(16 * hw - 16, dtype=torch.uint8)),
           dict(gamma_out=torch.zeros(32 * hw, dtype=torch.uint8)),          # the FP32 size for an FP16 guide
           dict(samples=dict(alloc_samples(2, hw, device="cpu"), wx=torch.zeros(hw))),
           dict(samples=dict(alloc_samples(2, hw, device="cpu"), strategy=torch.zeros(2 * hw - 1, dtype=torch.uint8))),
           dict(samples={k: v for k, v in alloc_samples(2, hw, device="cpu").items() if k != "radiance"}),
           dict(img=torch.zeros(hw - 1)), dict(g0_prev=torch.zeros(4 * hw - 4))]
    for kw in bad:
        with pytest.raises(ValueError):
            call(**kw)
    # sizes right: only then does the binding look at devices (CPU tensors are refused)
    with pytest.raises(TypeError):
        call()
