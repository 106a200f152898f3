"""Noise pins: measured phase-error variances of the oracle's blind rotation
and key switching against the closed-form variances of the construction.

Blind rotation (words^2, one word = 2^-32): each CMux step with abar_i != 0
adds sum_r digit_r * e_r over the 2l rows, i.e. 2l * N * E[d^2] * var(e)
with digits uniform on [-Bg/2, Bg/2): E[d^2] = (Bg^2 - 1)/12 + 1/4; the
decomposition rounding adds at most 1e-4 of that and is neglected.
Key switching: each of the N*t digits is non-zero with probability
(base-1)/base and then adds one KSK noise of variance var(e_ks); rounding
a'_j to t*basebit bits adds sum_j S_j * (2^(32 - t*basebit))^2 / 12.
"""
import numpy as np

from conftest import center, np_negacyclic, oparams, trivial_rotation
from paper_2005_01945_gb300 import synth

M32 = 1 << 32
MU = 1 << 29


def test_blind_rotation_variance(orc, full_keys):
    p, P, kd, bk, ksk = full_keys
    rng = np.random.default_rng(41)
    cnt = 4
    abar = rng.integers(1, 2 * p.N, size=(cnt, p.n + 1)).astype(np.int32)
    acc = orc.blind_rotate(P, bk, abar)
    errs = []
    for g in range(cnt):
        m = (int((abar[g, :p.n].astype(np.int64) * kd.s).sum()) - int(abar[g, p.n])) % (2 * p.N)
        ph = (acc[g, 1].astype(np.int64) - np_negacyclic(kd.S, acc[g, 0]).astype(np.int64)) % M32
        errs.append(center(((ph - trivial_rotation(MU, p.N, m).astype(np.int64)) % M32).astype(np.uint32)))
    errs = np.concatenate(errs).astype(np.float64)
    Bg = 1 << p.bg_bit
    Ed2 = (Bg * Bg - 1) / 12 + 0.25
    var_e = kd.bk_noise.astype(np.float64).var()
    expected = p.n * (2 * p.l) * p.N * Ed2 * var_e
    measured = float((errs ** 2).mean())
    assert abs(errs.mean()) < 4 * np.sqrt(expected / errs.size)
    assert abs(measured / expected - 1) < 0.10, (measured, expected)


def test_keyswitch_variance(orc, full_keys):
    p, P, kd, bk, ksk = full_keys
    rng = np.random.default_rng(42)
    cnt = 2000
    big = rng.integers(0, M32, size=(cnt, p.N + 1), dtype=np.uint64).astype(np.uint32)
    out = orc.keyswitch(P, ksk, big)
    ph_in = (big[:, p.N].astype(np.int64) - (big[:, :p.N].astype(np.int64) * kd.S).sum(axis=1)) % M32
    ph_out = orc.phase(P, kd.s, out).astype(np.int64)
    err = center(((ph_out - ph_in) % M32).astype(np.uint32)).astype(np.float64)
    # With the key fixed, slot (j, q) adds -X with X uniform over the digit
    # values {0, e_1, .., e_(base-1)} of its KSK noise: the error has mean
    # -sum m_s and variance sum var_s plus the rounding term.
    e = kd.ksk_noise.astype(np.float64)
    ez = np.concatenate([np.zeros(e.shape[:2] + (1,)), e], axis=2)
    mean_exp = -ez.mean(axis=2).sum()
    var_exp = ez.var(axis=2).sum() + kd.S.sum() * (2.0 ** (32 - p.ks_t * p.ks_basebit)) ** 2 / 12
    assert abs(err.mean() - mean_exp) < 4 * np.sqrt(var_exp / cnt)
    assert abs(err.var() / var_exp - 1) < 0.12, (err.var(), var_exp)
    # averaged over keys the variance is N t (base-1)/base var(e) (closed form)
    base = 1 << p.ks_basebit
    nominal = p.N * p.ks_t * (base - 1) / base * e.var()
    assert abs((ez.var(axis=2).sum() + np.square(ez.mean(axis=2)).sum()) / nominal - 1) < 0.05
