"""Pins for encryption and key generation: every phase is checked against
its exact expected value with an independent numpy phase computation."""
import numpy as np

from conftest import center, np_negacyclic, oparams, toy_params
from paper_2005_01945_gb300 import synth

M32 = 1 << 32


def test_encrypt_phase_is_message_plus_noise(orc):
    p = synth.TFHEParams()
    P = oparams(p)
    kd = synth.key_draws(p, 11)
    bits = synth.random_bits(1000, 11, "enc")
    cd = synth.ct_draws(p, 1000, 11, "enc")
    ct = orc.encrypt_bits(P, kd.s, cd.mask, cd.noise, bits)
    # independent phase: b - a.s computed with Python-int dot products
    a = ct[:, :p.n].astype(np.int64)
    ph = (ct[:, p.n].astype(np.int64) - (a * kd.s.astype(np.int64)).sum(axis=1)) % M32
    mu = np.where(bits == 1, 1 << 29, M32 - (1 << 29))
    assert np.array_equal(ph, (mu + cd.noise.astype(np.int64)) % M32)
    assert np.array_equal(orc.phase(P, kd.s, ct), ph.astype(np.uint32))
    assert np.array_equal(orc.decrypt_bits(P, kd.s, ct), bits)


def test_bootstrapping_key_rows(orc):
    """Row r = c*l + j of BK_i: body row (c=1) has phase e + s_i h_j X^0;
    mask row (c=0) has its mask raised by s_i h_j, so its phase is
    e - s_i h_j S(X)."""
    p = toy_params(n=6, N=32)
    P = oparams(p)
    kd = synth.key_draws(p, 5)
    bk = orc.keygen_bk(P, kd.s, kd.S, kd.bk_mask, kd.bk_noise)
    for i in range(p.n):
        for r in range(2 * p.l):
            c, j = divmod(r, p.l)
            h = 1 << (32 - p.bg_bit * (j + 1))
            a, b = bk[i, r, 0], bk[i, r, 1]
            phase = (b.astype(np.int64) - np_negacyclic(kd.S, a).astype(np.int64)) % M32
            want = kd.bk_noise[i, r].astype(np.int64)
            if c == 1:
                want = want.copy()
                want[0] += int(kd.s[i]) * h
            else:
                want = want - int(kd.s[i]) * h * kd.S.astype(np.int64)
            assert np.array_equal(phase, want % M32), (i, r)


def test_keyswitching_key_rows(orc):
    p = toy_params(n=10, N=16)
    P = oparams(p)
    kd = synth.key_draws(p, 6)
    ksk = orc.keygen_ksk(P, kd.s, kd.S, kd.ksk_mask, kd.ksk_noise)
    for j in range(p.N):
        for q in range(p.ks_t):
            for d in range(1, 4):
                row = ksk[j, q, d - 1]
                ph = (int(row[p.n]) - int((row[:p.n].astype(np.int64) * kd.s).sum())) % M32
                want = (d * int(kd.S[j]) * (1 << (32 - 2 * (q + 1))) + int(kd.ksk_noise[j, q, d - 1])) % M32
                assert ph == want


def test_noise_draws_have_stated_sigma():
    p = synth.TFHEParams()
    kd = synth.key_draws(p, 9)
    sd_bk = kd.bk_noise.astype(np.float64).std() / 2.0 ** 32
    sd_ks = kd.ksk_noise.astype(np.float64).std() / 2.0 ** 32
    assert abs(sd_bk / p.sigma_bk - 1) < 0.01
    assert abs(sd_ks / p.sigma_lwe - 1) < 0.02
