"""Pin for the oracle's evaluation order: the gates of a circuit run as tasks
ordered only by the ciphertext rows they read and write, so the result must
not depend on how many threads run them.  Every circuit kind is evaluated
with one thread (the gates run one by one in the order the circuit code
creates them) and with eight (independent gates run side by side, in any
order the dependences allow); every output word must agree.  A missing or
wrong dependence would let a gate read a row before it is written, or
after it is overwritten, and change the ciphertexts."""
import numpy as np
import pytest

from conftest import oparams, toy_params
from paper_2005_01945_gb300 import synth


@pytest.fixture(scope="module")
def toy(orc):
    p = toy_params(n=8, N=32)
    P = oparams(p)
    kd = synth.key_draws(p, 57)
    bk = orc.keygen_bk(P, kd.s, kd.S, kd.bk_mask, kd.bk_noise)
    ksk = orc.keygen_ksk(P, kd.s, kd.S, kd.ksk_mask, kd.ksk_noise)
    return p, P, kd, bk, ksk


def _enc(orc, p, P, kd, xs, w, tag):
    bits = synth.to_bits(xs, w)
    cd = synth.ct_draws(p, bits.shape, 58, tag)
    return orc.encrypt_bits(P, kd.s, cd.mask, cd.noise, bits)


@pytest.mark.parametrize("name,w,batch", [
    ("add", 9, 3), ("mul", 7, 2), ("add_maj", 9, 2), ("add_nw", 6, 2), ("mul_tree", 7, 2),
    ("mul_tree_maj", 6, 2), ("add_prefix", 13, 2), ("mul_dadda", 9, 2), ("mul_full", 6, 2),
    ("mul_karatsuba", 10, 1)])
def test_circuit_result_independent_of_threads(orc, toy, name, w, batch):
    p, P, kd, bk, ksk = toy
    a, b = synth.int_pairs(batch, w, 59, name)
    A, B = _enc(orc, p, P, kd, a, w, name + "a"), _enc(orc, p, P, kd, b, w, name + "b")
    fn = getattr(orc, name)
    r1, g1 = fn(P, bk, ksk, w, A, B, nthreads=1)
    r8, g8 = fn(P, bk, ksk, w, A, B, nthreads=8)
    assert g1 == g8
    assert np.array_equal(r1, r8)


def test_matvec_independent_of_threads(orc, toy):
    p, P, kd, bk, ksk = toy
    w, rows, cols = 4, 2, 5
    M = synth.random_uints((rows, cols), w, 60, "M")
    v = synth.random_uints(cols, w, 60, "v")
    oM, ov = _enc(orc, p, P, kd, M, w, "M"), _enc(orc, p, P, kd, v, w, "v")
    y1, g1 = orc.matvec(P, bk, ksk, w, oM, ov, nthreads=1)
    y8, g8 = orc.matvec(P, bk, ksk, w, oM, ov, nthreads=8)
    assert g1 == g8
    assert np.array_equal(y1, y8)
    dec = synth.from_bits(orc.decrypt_bits(P, kd.s, y8))
    assert np.array_equal(dec, (M * v[None, :]).sum(axis=1) % (1 << w))
