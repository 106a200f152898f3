"""Noise of the GPU path against the closed forms of the construction.

20,000 gates with fresh inputs: the output phase error (phase - (+-1/8))
must have the mean and variance predicted from the key's noise draws:
  blind rotation: every CMux step with abar_i != 0 adds
      sum_r digit_r * e_r: variance 2l N E[d^2] var(e_bk), digits uniform on
      [-Bg/2, Bg/2): E[d^2] = (Bg^2 - 1)/12 + 1/4;
  key switching with the fixed key: mean -sum_s m_s, variance
      sum_s var_s + sum_j S_j (2^(32 - t basebit))^2 / 12 (see the oracle's
      noise pin for the derivation).
Every output decrypts correctly and the worst error keeps its margin.
"""
import numpy as np
import pytest

from paper_2005_01945_gb300 import synth

pytestmark = pytest.mark.gpu


def test_output_noise_matches_closed_form():
    import torch
    from paper_2005_01945_gb300 import api, build
    build.build()
    p = synth.TFHEParams()
    kd = synth.key_draws(p, 2024)
    d = api.to_device
    bk, ksk = api.keygen(p, d(kd.s), d(kd.S), d(kd.bk_mask), d(kd.bk_noise), d(kd.ksk_mask),
                         d(kd.ksk_noise))
    ctx = api.Context(p)
    ctx.set_keys(bk, ksk)
    count = 20000
    bits = synth.random_bits((2, count), 5, "noise")
    cd = synth.ct_draws(p, (2, count), 5, "noise")
    s_dev = d(kd.s)
    a = api.encrypt_bits(p, s_dev, d(cd.mask[0]), d(cd.noise[0]), d(bits[0]))
    b = api.encrypt_bits(p, s_dev, d(cd.mask[1]), d(cd.noise[1]), d(bits[1]))
    ops = synth._gen(5, "noise_ops").integers(0, 6, size=count).astype(np.uint8)
    out = torch.empty((count, api.LWE_STRIDE), dtype=torch.int32, device="cuda")
    ctx.bootstrap_gates(d(ops), a, b, out)
    ph = api.phase(p, s_dev, out).cpu().numpy().astype(np.int64)
    x, y = bits[0].astype(int), bits[1].astype(int)
    truth = np.select([ops == 0, ops == 1, ops == 2, ops == 3, ops == 4, ops == 5],
                      [1 - (x & y), x & y, x | y, x ^ y, 1 - (x | y), 1 - (x ^ y)])
    ideal = np.where(truth == 1, 1 << 29, -(1 << 29))
    err = (ph - ideal).astype(np.float64)

    Bg = 1 << p.bg_bit
    Ed2 = (Bg * Bg - 1) / 12 + 0.25
    var_br = p.n * (1 - 1 / (2 * p.N)) * 2 * p.l * p.N * Ed2 * kd.bk_noise.astype(np.float64).var()
    e = kd.ksk_noise.astype(np.float64)
    ez = np.concatenate([np.zeros(e.shape[:2] + (1,)), e], axis=2)
    mean_ks = -ez.mean(axis=2).sum()
    var_ks = ez.var(axis=2).sum() + kd.S.sum() * (2.0 ** (32 - p.ks_t * p.ks_basebit)) ** 2 / 12
    var_exp = var_br + var_ks
    assert abs(err.mean() - mean_ks) < 5 * np.sqrt(var_exp / count)
    assert abs(err.var() / var_exp - 1) < 0.05, (err.var(), var_exp)
    assert np.array_equal((ph > 0).astype(int), truth)
    assert np.abs(err).max() < (1 << 29) / 2      # margin 1/8 > 2 x worst error
    ctx.close()
