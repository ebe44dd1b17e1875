"""The EM step keeps a small covariance where a frame's mass dwarfs the stored
guide's (Sec. 3.2's weighted stepwise EM with lambda = eta a / A -> 1), and
where one bright draw follows a dim one elsewhere. In binary32, 1 - lambda
formed as a difference, or the covariance formed as lambda M2 -
(lambda delta)^2 from moments about a fixed point, loses most of such a
covariance; the kernels' mixture form (West's incremental mean and central
moment, 1 - lambda = (1 - eta) pi M0 / A) keeps it. Checked through the
staged calls on BF16 storage (its 8-bit significand spans the tiny
covariances that FP16 would flush and FP32's raw moments would bury): every
field within one storage ulp of the oracle's FP64 step rounded once."""
import numpy as np
import pytest

import oracle as O
from paper_2112_09728_gb300 import scenes

from _pg import dev, guide, host, ocam, ocfg
from test_gpu_precision import _central_to_raw_moments, _raw_to_central, _record_bytes, _records_to_central, \
    _round, _ulp

pytestmark = pytest.mark.gpu


def _case():
    """64 Lambertian pixels with normal +z under a top-down camera: stored
    masses W from 1e-2 down to 1e-9 (so that 1 - lambda spans 1e-2 to 1e-9),
    two prior covariance scales, and four sample sets of two draws: one
    training draw; two BRDF draws 1e-3 apart with radiances 1e-3 then 1e3;
    the same 0.1 apart; two equal draws 0.02 apart."""
    W, H, spp = 16, 4, 2
    hw = W * H
    par = scenes.Params(W, H, spp=spp, seed=77)
    g0 = np.tile(np.array([[0.0, 0.0, 1.0, 1.0]], np.float32), (hw, 1))
    g1 = np.tile(np.array([[0.0, 0.0, -1.0, 0.8]], np.float32), (hw, 1))
    p = np.arange(hw)
    e, kind = p % 8, (p // 8) % 4
    sxx = np.where(p < 32, 1e-3, 1e-5)
    central = np.zeros((hw, 8))
    central[:, 0], central[:, 1] = 0.47, 0.53
    central[:, 2], central[:, 3] = sxx, 1.3 * sxx
    central[:, 4] = 0.3 * np.sqrt(central[:, 2] * central[:, 3])
    central[:, 5], central[:, 6], central[:, 7] = 0.5, 3.0, 10.0 ** (-2.0 - e)
    central = _round(central, "bf16")            # the stored prior, exactly
    # the first draw about two standard deviations of the guide (as its density
    # sees it, the variance floored at 1e-4) from the mean
    u0 = central[:, :2] + 2.0 * np.sqrt(np.maximum(sxx, 1e-4))[:, None] * np.array([1.0, -0.7])
    off = np.select([kind == 1, kind == 2, kind == 3], [1e-3, 0.1, 0.02], 0.0)
    u1 = u0 + np.stack([off, 0.5 * off], 1)
    L0 = np.where((kind == 1) | (kind == 2), 1e-3, 1.0)
    L1 = np.where((kind == 1) | (kind == 2), 1e3, 1.0)
    d0, d1 = O.square_to_hemi(u0), O.square_to_hemi(u1)
    d = np.concatenate([d0, d1]).astype(np.float32)
    strat = np.concatenate([np.zeros(hw, np.uint8), np.where(kind == 0, 1, 0).astype(np.uint8)])
    samples = dict(wx=d[:, 0].copy(), wy=d[:, 1].copy(), wz=d[:, 2].copy(),
                   radiance=np.concatenate([L0, L1]).astype(np.float32),
                   estimate=np.zeros(spp * hw, np.float32), strategy=strat)
    return par, g0, g1, central, samples


def test_em_step_keeps_a_small_covariance_as_lambda_tends_to_one():
    par, g0, g1, central, samples = _case()
    cam = scenes.top_down_camera()
    gp = guide(par, "bf16")
    gp.pg_set_gamma(dev(_record_bytes(central, "bf16")))
    gp.pg_reproject(dev(g0), dev(g1), cam, dev(g0))
    gp.pg_update(dev(g0), dev(g1), cam, {k: dev(v) for k, v in samples.items()})
    got = _records_to_central(host(gp.pg_get_gamma()), "bf16")
    gp.close()
    ref = O.update(ocfg(par), ocam(cam), g0, g1, _central_to_raw_moments(central),
                   {k: (v.astype(np.float64) if v.dtype != np.uint8 else v) for k, v in samples.items()})
    ref = _raw_to_central(ref)
    # the step moved every guide, and the covariances it left span 1e-12 to 1e-3
    assert (np.abs(ref[:, :2] - central[:, :2]).max(1) > 5e-4).all()
    assert ref[:, 2].min() < 1e-11 and ref[:, 2].max() > 1e-4
    r16 = _round(ref, "bf16")
    ulps = np.abs(got - r16) / _ulp(r16, "bf16")
    assert (got[:, 6] == r16[:, 6]).all()
    assert (ulps <= 1.01).all(), ("worst ulps per field", ulps.max(0), "pixels", np.nonzero((ulps > 1.01).any(1))[0])
