"""The Adam optimiser state of the differentiable form: BF16 moments stored
with stochastic rounding, and checkpoint/resume of the moments.

* BF16 moments: each step's m and v are the oracle's FP64 step from the
  previous stored moments, rounded stochastically by the rule written out in
  test_gpu_precision (from its definition) with the oracle's Philox words at
  counters (pixel, step, 0, 6) and (pixel, step, 1, 6). The oracle's
  trajectory carries its own rounded moments; the GPU's are compared with it
  element by element. A stored moment may differ by a BF16 ulp where the
  binary32 and FP64 values straddle the random threshold (chance ~1e-5),
  and by up to two in the steps after; such pixels are counted and left out
  of the Gamma comparison, which
  otherwise keeps the FP32-moment tolerance (1e-5 relative + 1e-6).
* The rounding is what keeps v moving: with beta2 = 0.999 an update is a
  thousandth of v, below BF16's half ulp once v passes a third of g^2, so
  round-to-nearest stalls there (emulated here on the CPU) while the GPU's
  stochastically rounded v tracks (1 - beta2^t) g^2 on average.
* Checkpoint/resume: moments got from one context and set into a fresh one
  continue bit-identically.
"""
import numpy as np
import pytest

import oracle as O
from paper_2112_09728_gb300 import scenes

from _pg import close, dev, get_gamma_rows, guide, host, ocfg, set_gamma_rows
from test_gpu_precision import _round, _sr_reference, _ulp

pytestmark = pytest.mark.gpu


def _case(seed, W=37, H=21):
    rng = np.random.default_rng(seed)
    par = scenes.Params(W, H, seed=seed * 17 + 3)
    gam = scenes.random_gamma(rng, W * H, k_hi=32)
    return rng, par, gam


def _moment_bits(cfg, step, hw):
    """16 random bits per moment: [hw, 12] (m_0..m_5, v_0..v_5)."""
    words = []
    for call in (0, 1):
        ctr = np.zeros((hw, 4), np.uint32)
        ctr[:, 0] = np.arange(hw)
        ctr[:, 1] = step
        ctr[:, 2] = call
        ctr[:, 3] = 6
        words.append(O.philox(ctr, (cfg.seed_lo, cfg.seed_hi)).astype(np.int64))
    w = np.concatenate(words, 1)
    return np.stack([(w[:, n // 2] >> (16 * (n % 2))) & 0xFFFF for n in range(12)], 1)


def _grad(rng, hw):
    return rng.normal(size=(hw, 6)).astype(np.float32) * np.array([1, 1, 50, 50, 50, 1], np.float32)


# the C ABI takes the hyper-parameters as binary32; the oracle gets the same
# values (1 - beta2 differs by 1.3e-5 relative between 0.999 and 0.999f, a
# visible fraction of a BF16 ulp)
LR, B1, B2, EPS = (float(np.float32(x)) for x in (1e-2, 0.9, 0.999, 1e-8))


def test_bf16_moments_follow_the_oracle_with_stochastic_rounding():
    rng, par, gam = _case(71)
    hw = par.width * par.height
    gp = guide(par, adam_dtype="bf16")
    set_gamma_rows(gp, gam)
    cfg = ocfg(par)
    ref = gam.astype(np.float64)
    m = v = np.zeros((hw, 6))
    flipped = np.zeros(hw, bool)
    for step in range(1, 6):
        grad = _grad(rng, hw)
        gp.pg_adam_step(dev(np.ascontiguousarray(grad.T)), lr=LR, beta1=B1, beta2=B2, eps=EPS, step=step)
        ref, m64, v64 = O.adam(cfg, ref, grad.astype(np.float64), m, v, LR, B1, B2, EPS, step)
        bits = _moment_bits(cfg, step, hw)
        m = _sr_reference(m64, bits[:, :6], "bf16")
        v = _sr_reference(v64, bits[:, 6:], "bf16")
        gm, gv = (host(t).T.astype(np.float64) for t in gp.pg_get_adam_state())
        for got, want in ((gm, m), (gv, v)):
            assert (np.abs(got - want) <= 2.01 * _ulp(want, "bf16")).all()
            flipped |= (got != want).any(1)
        # the rounding is live: about a quarter of the moments round away from nearest
        rn = _round(m64, "bf16")
        assert (m != rn).mean() > 0.15
    assert flipped.mean() < 0.01
    got = get_gamma_rows(gp)
    assert close(got[~flipped], ref[~flipped], 1e-5, 1e-6) <= 1.0


def test_bf16_second_moment_tracks_where_round_to_nearest_stalls():
    import torch
    W, H, steps = 32, 32, 1500
    hw = W * H
    rng = np.random.default_rng(72)
    par = scenes.Params(W, H, seed=99)
    gp = guide(par, adam_dtype="bf16")
    g = (rng.uniform(0.5, 2.0, (6, hw)) * rng.choice([-1.0, 1.0], (6, hw))).astype(np.float32)
    G = dev(g)
    for t in range(1, steps + 1):
        gp.pg_adam_step(G, lr=1e-4, step=t)
    m, v = (host(x).astype(np.float64) for x in gp.pg_get_adam_state())
    g64 = g.astype(np.float64)
    v_exact = (1 - 0.999 ** steps) * g64 * g64
    m_exact = (1 - 0.9 ** steps) * g64
    # per element the rounding noise of v is a few percent; the mean over 6144 is unbiased
    assert abs((v / v_exact).mean() - 1) < 5e-3
    assert abs((m / m_exact).mean() - 1) < 5e-3
    assert np.abs(v / v_exact - 1).max() < 0.25
    # round to nearest in BF16 with the same binary32 arithmetic stalls near g^2 / 3
    b2 = torch.tensor(0.999, dtype=torch.float32)
    vr = torch.zeros(6 * hw, dtype=torch.bfloat16)
    gg = torch.from_numpy(g.ravel())
    c = (1 - b2) * gg * gg
    for _ in range(steps):
        vr = (b2 * vr.float() + c).to(torch.bfloat16)
    stalled = vr.double().numpy().reshape(6, hw) / v_exact
    assert stalled.mean() < 0.75
    assert torch.isfinite(gp.pg_gamma_to_f32()).all()


@pytest.mark.parametrize("adam_dtype", ["f32", "bf16"])
def test_adam_state_checkpoint_resume_is_bit_identical(adam_dtype):
    import torch
    rng, par, gam = _case(73)
    hw = par.width * par.height
    grads = [dev(np.ascontiguousarray(_grad(rng, hw).T)) for _ in range(5)]
    a = guide(par, gamma_dtype="f16", adam_dtype=adam_dtype)
    set_gamma_rows(a, gam)
    for t in range(3):
        a.pg_adam_step(grads[t], lr=1e-2, step=t + 1)
    gam_ck = a.pg_get_gamma().clone()
    m_ck, v_ck = (x.clone() for x in a.pg_get_adam_state())
    b = guide(par, gamma_dtype="f16", adam_dtype=adam_dtype)
    with pytest.raises(RuntimeError):
        b.pg_get_adam_state()                       # no state before a step or a set
    b.pg_set_gamma(gam_ck)
    b.pg_set_adam_state(m_ck, v_ck)
    for t in (3, 4):
        a.pg_adam_step(grads[t], lr=1e-2, step=t + 1)
        b.pg_adam_step(grads[t], lr=1e-2, step=t + 1)
    assert torch.equal(a.pg_get_gamma(), b.pg_get_gamma())
    for x, y in zip(a.pg_get_adam_state(), b.pg_get_adam_state()):
        assert torch.equal(x, y)
    if adam_dtype == "bf16":
        m, _ = a.pg_get_adam_state()
        assert torch.equal(m, m.to(torch.bfloat16).float())     # stored in BF16
