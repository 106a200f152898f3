"""Pins for the oracle's bootstrapping chain: blind rotation, sample
extraction, key switching, gate combine and whole gates.

Exact pins use noiseless keys, where the scheme's output is a closed form:
with trivial (zero-mask, zero-noise) bootstrapping keys the accumulator is
exactly (0, X^(sum abar_i s_i - bbar) v); extraction is an exact phase
identity; a noiseless key switch of inputs on the 2^-16 grid is exact.
"""
import numpy as np
import pytest

from conftest import center, np_negacyclic, oparams, toy_params, trivial_rotation
from paper_2005_01945_gb300 import synth

M32 = 1 << 32
MU = 1 << 29


def _keys(orc, p, seed, **kw):
    P = oparams(p)
    kd = synth.key_draws(p, seed, **kw)
    bk = orc.keygen_bk(P, kd.s, kd.S, kd.bk_mask, kd.bk_noise)
    ksk = orc.keygen_ksk(P, kd.s, kd.S, kd.ksk_mask, kd.ksk_noise)
    return P, kd, bk, ksk


def _expected_rotation(p, kd, abar):
    return (int((abar[:p.n].astype(np.int64) * kd.s).sum()) - int(abar[p.n])) % (2 * p.N)


def test_blind_rotation_trivial_keys_every_rotation_toy(orc):
    """All 2N values of bbar, random abar: acc = (0, X^m v) exactly."""
    p = toy_params(n=8, N=32)
    P, kd, bk, _ = _keys(orc, p, 21, noiseless=True, zero_bk_mask=True)
    rng = np.random.default_rng(0)
    abar = np.zeros((2 * p.N, p.n + 1), np.int32)
    abar[:, :p.n] = rng.integers(0, 2 * p.N, size=(2 * p.N, p.n))
    abar[:, p.n] = np.arange(2 * p.N)
    acc = orc.blind_rotate(P, bk, abar)
    for g in range(2 * p.N):
        m = _expected_rotation(p, kd, abar[g])
        assert not acc[g, 0].any()
        assert np.array_equal(acc[g, 1], trivial_rotation(MU, p.N, m)), g


def test_blind_rotation_trivial_keys_full_size(orc):
    p = synth.TFHEParams()
    P, kd, bk, _ = _keys(orc, p, 22, noiseless=True, zero_bk_mask=True)
    rng = np.random.default_rng(1)
    abar = rng.integers(0, 2 * p.N, size=(2, p.n + 1)).astype(np.int32)
    abar[1, :10] = 0      # a few skipped steps (abar_i = 0)
    acc = orc.blind_rotate(P, bk, abar)
    for g in range(2):
        m = _expected_rotation(p, kd, abar[g])
        assert not acc[g, 0].any()
        assert np.array_equal(acc[g, 1], trivial_rotation(MU, p.N, m))


def test_blind_rotation_noiseless_random_masks_bound(orc):
    """Zero noise, uniform masks: every coefficient of the accumulator's
    phase equals the closed form up to the decomposition rounding, at most
    (N + 1) * 2^11 per CMux step whose key bit is 1."""
    p = toy_params(n=8, N=32)
    P, kd, bk, _ = _keys(orc, p, 23, noiseless=True)
    rng = np.random.default_rng(2)
    abar = rng.integers(0, 2 * p.N, size=(64, p.n + 1)).astype(np.int32)
    acc = orc.blind_rotate(P, bk, abar)
    for g in range(64):
        m = _expected_rotation(p, kd, abar[g])
        phase = (acc[g, 1].astype(np.int64) - np_negacyclic(kd.S, acc[g, 0]).astype(np.int64)) % M32
        err = center(((phase - trivial_rotation(MU, p.N, m).astype(np.int64)) % M32).astype(np.uint32))
        steps = int(((abar[g, :p.n] != 0) & (kd.s == 1)).sum())
        assert np.abs(err).max() <= steps * (p.N + 1) * (1 << 11)


def test_sample_extraction_phase_identity(orc):
    p = synth.TFHEParams()
    P = oparams(p)
    rng = np.random.default_rng(3)
    S = rng.integers(0, 2, size=p.N).astype(np.int32)
    for _ in range(4):
        acc = rng.integers(0, M32, size=(2, p.N), dtype=np.uint64).astype(np.uint32)
        tlwe_phase0 = (int(acc[1, 0]) - int(np_negacyclic(S, acc[0])[0])) % M32
        big = orc.sample_extract(P, acc)
        lwe_phase = (int(big[p.N]) - int((big[:p.N].astype(np.int64) * S).sum())) % M32
        assert lwe_phase == tlwe_phase0


@pytest.mark.parametrize("full", [False, True])
def test_keyswitch_noiseless(orc, full):
    p = synth.TFHEParams() if full else toy_params(n=16, N=64)
    P, kd, _, ksk = _keys(orc, p, 24, noiseless=True)
    rng = np.random.default_rng(4)
    cnt = 8
    big = rng.integers(0, M32, size=(cnt, p.N + 1), dtype=np.uint64).astype(np.uint32)
    grid = big.copy()
    grid[:, :p.N] &= np.uint32(0xFFFF0000)       # a'_j on the 2^-16 grid: exact
    for x, exact in ((grid, True), (big, False)):
        out = orc.keyswitch(P, ksk, x)
        ph_in = (x[:, p.N].astype(np.int64) - (x[:, :p.N].astype(np.int64) * kd.S).sum(axis=1)) % M32
        ph_out = orc.phase(P, kd.s, out).astype(np.int64)
        err = center(((ph_out - ph_in) % M32).astype(np.uint32))
        if exact:
            assert not err.any()
        else:
            assert np.abs(err).max() <= int(kd.S.sum()) * (1 << 15)


GATES = {0: "NAND", 1: "AND", 2: "OR", 3: "XOR", 4: "NOR", 5: "XNOR", 7: "ANDNY", 8: "ANDYN",
         9: "ORNY", 10: "ORYN"}


def _truth_tables():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "gate_truth_tables.txt")
    tab = {}
    for line in open(path):
        line = line.split("#")[0].split()
        if len(line) in (5, 9):
            tab[line[0]] = [int(v) for v in line[1:]]
    return tab


def test_gate_combine_noiseless_signs(orc):
    """Noiseless inputs of phase exactly +-1/8: the combined phase has the
    sign of the gate's truth value with a margin of at least 1/8."""
    p = toy_params(n=16, N=64)
    P = oparams(p)
    kd = synth.key_draws(p, 25)
    tt = _truth_tables()
    a_bits = np.array([0, 0, 1, 1], np.uint8)
    b_bits = np.array([0, 1, 0, 1], np.uint8)
    cd = synth.ct_draws(p, (2, 4), 25, "comb", noiseless=True)
    ca = orc.encrypt_bits(P, kd.s, cd.mask[0], cd.noise[0], a_bits)
    cb = orc.encrypt_bits(P, kd.s, cd.mask[1], cd.noise[1], b_bits)
    for op, name in GATES.items():
        for k in range(4):
            c = orc.gate_combine(P, op, ca[k], cb[k])
            ph = int(center(orc.phase(P, kd.s, c[None])[0]))
            assert (ph > 0) == bool(tt[name][k]), (name, k)
            assert abs(ph) >= MU


def test_bootstrap_toy_all_phase_octants(orc):
    """Whole chain on toy parameters: a noiseless input of phase (2k+1)/16
    bootstraps to +1/8 iff the phase lies in [0, 1/2)."""
    p = toy_params(n=8, N=64)
    P, kd, bk, ksk = _keys(orc, p, 26)
    rng = np.random.default_rng(5)
    phases = np.array([(2 * k + 1) * (M32 // 16) for k in range(8)] * 4, dtype=np.uint64)
    mask = rng.integers(0, M32, size=(len(phases), p.n), dtype=np.uint64)
    ct = np.zeros((len(phases), p.n + 1), np.uint32)
    ct[:, :p.n] = mask
    ct[:, p.n] = ((mask * kd.s.astype(np.uint64)).sum(axis=1) + phases) % M32
    out = orc.bootstrap(P, bk, ksk, ct)
    ph = center(orc.phase(P, kd.s, out))
    want = np.where(phases < M32 // 2, MU, -MU)
    # key-switch noise dominates: sigma ~ sqrt(N t 3/4) 2^17 ~ 2.6e6 words here
    assert np.abs(ph - want).max() < (1 << 25)


def test_gates_full_parameters_truth_tables(orc, full_keys):
    """Every gate on every input pair at the full parameter set."""
    p, P, kd, bk, ksk = full_keys
    tt = _truth_tables()
    ops = np.repeat(np.array(sorted(GATES), dtype=np.uint8), 4)
    a_bits = np.tile(np.array([0, 0, 1, 1], np.uint8), len(GATES))
    b_bits = np.tile(np.array([0, 1, 0, 1], np.uint8), len(GATES))
    cd = synth.ct_draws(p, (2, len(ops)), 27, "tt")
    ca = orc.encrypt_bits(P, kd.s, cd.mask[0], cd.noise[0], a_bits)
    cb = orc.encrypt_bits(P, kd.s, cd.mask[1], cd.noise[1], b_bits)
    out = orc.gates(P, bk, ksk, ops, ca, cb)
    got = orc.decrypt_bits(P, kd.s, out)
    want = np.array([tt[GATES[int(o)]][k % 4] for k, o in enumerate(ops)], np.uint8)
    assert np.array_equal(got, want)
    # fresh output noise is far below the 1/8 decision margin
    ph = center(orc.phase(P, kd.s, out))
    assert np.abs(np.abs(ph) - MU).max() < MU // 4


def test_majority_gate_truth_table_and_margin(orc, full_keys):
    """MAJ: noiseless combined phases are +-1/8 or +-3/8 with the sign of the
    majority; bootstrapped at full parameters it decrypts to the table."""
    p, P, kd, bk, ksk = full_keys
    tt = _truth_tables()["MAJ3"]
    bits = np.array([[(k >> 2) & 1, (k >> 1) & 1, k & 1] for k in range(8)], np.uint8).T
    cd = synth.ct_draws(p, (3, 8), 28, "maj", noiseless=True)
    c = [orc.encrypt_bits(P, kd.s, cd.mask[i], cd.noise[i], bits[i]) for i in range(3)]
    for k in range(8):
        comb = orc.gate_combine3(P, orc.MAJ, c[0][k], c[1][k], c[2][k])
        ph = int(center(orc.phase(P, kd.s, comb[None])[0]))
        assert (ph > 0) == bool(tt[k]) and abs(ph) >= MU
    cdn = synth.ct_draws(p, (3, 8), 29, "majn")
    cn = [orc.encrypt_bits(P, kd.s, cdn.mask[i], cdn.noise[i], bits[i]) for i in range(3)]
    out = np.stack([orc.gate3(P, bk, ksk, orc.MAJ, cn[0][k], cn[1][k], cn[2][k]) for k in range(8)])
    assert orc.decrypt_bits(P, kd.s, out).tolist() == tt
