"""GPU parity of the circuit schedules through the C ABI.

Bit-exact comparisons with the oracle use the real ring (N = 1024, same
gadget and key switch) with LWE dimension n = 16, which the library takes
at runtime; the oracle's bootstrap is then ~30x cheaper, so every circuit
kind can be compared word for word.  The full-size workloads at n = 500
(256 32-bit additions, 64 + 64 multiplications, the 16x16 matvec) are run
as one schedule each, exactly as the benchmark runs them; every output is
checked by decryption, and sampled whole instances (16 additions, one
16-bit and one 32-bit multiplication, one matvec output row) are
recomputed by the oracle gate by gate and compared word for word.
"""
import numpy as np
import pytest

from conftest import oparams
from paper_2005_01945_gb300 import synth

pytestmark = pytest.mark.gpu


class Env:
    def __init__(self, orc, n, seed):
        import torch
        from paper_2005_01945_gb300 import api, build
        build.build()
        self.torch, self.api, self.orc = torch, api, orc
        self.p = synth.TFHEParams(n=n)
        self.P = oparams(self.p)
        self.kd = synth.key_draws(self.p, seed)
        d = api.to_device
        kd = self.kd
        bk, ksk = api.keygen(self.p, d(kd.s), d(kd.S), d(kd.bk_mask), d(kd.bk_noise),
                             d(kd.ksk_mask), d(kd.ksk_noise))
        self.ctx = api.Context(self.p)
        self.ctx.set_keys(bk, ksk)
        self.s_dev = d(kd.s)
        self.obk = orc.keygen_bk(self.P, kd.s, kd.S, kd.bk_mask, kd.bk_noise)
        self.oksk = orc.keygen_ksk(self.P, kd.s, kd.S, kd.ksk_mask, kd.ksk_noise)

    def enc_ints(self, xs, w, seed, tag):
        """integers -> (device [..., w, 512], oracle [..., w, n+1])"""
        bits = synth.to_bits(xs, w)
        cd = synth.ct_draws(self.p, bits.shape, seed, tag)
        o = self.orc.encrypt_bits(self.P, self.kd.s, cd.mask, cd.noise, bits)
        d = self.api.encrypt_bits(self.p, self.s_dev, self.api.to_device(cd.mask),
                                  self.api.to_device(cd.noise), self.api.to_device(bits))
        return d, o

    def out(self, shape):
        return self.torch.zeros(tuple(shape) + (512,), dtype=self.torch.int32, device="cuda")

    def host(self, t):
        return t.cpu().numpy().view(np.uint32)[..., :self.p.n + 1]

    def dec_ints(self, o):
        return synth.from_bits(self.orc.decrypt_bits(self.P, self.kd.s, o))


@pytest.fixture(scope="module")
def small(orc):
    e = Env(orc, 16, 61)
    yield e
    e.ctx.close()


@pytest.mark.parametrize("w,batch", [(1, 3), (2, 3), (5, 3), (32, 2)])
def test_add_bit_exact(small, w, batch):
    E = small
    a, b = synth.int_pairs(batch, w, 1, f"add{w}")
    da, oa = E.enc_ints(a, w, 2, f"a{w}")
    db, ob = E.enc_ints(b, w, 2, f"b{w}")
    R = E.out((batch, w))
    E.ctx.add_n(w, da, db, R)
    want, gates = E.orc.add(E.P, E.obk, E.oksk, w, oa, ob)
    got = E.host(R)
    assert np.array_equal(got, want)
    assert np.array_equal(E.dec_ints(got), (a + b) % (1 << w))
    assert E.ctx.status() == 0


@pytest.mark.parametrize("w,batch", [(1, 2), (3, 2), (8, 2)])
def test_mul_bit_exact(small, w, batch):
    E = small
    a, b = synth.int_pairs(batch, w, 3, f"mul{w}")
    da, oa = E.enc_ints(a, w, 4, f"ma{w}")
    db, ob = E.enc_ints(b, w, 4, f"mb{w}")
    R = E.out((batch, w))
    E.ctx.mul_n(w, da, db, R)
    want, _ = E.orc.mul(E.P, E.obk, E.oksk, w, oa, ob)
    got = E.host(R)
    assert np.array_equal(got, want)
    assert np.array_equal(E.dec_ints(got), (a * b) % (1 << w))


def test_matvec_bit_exact(small):
    E = small
    w, rows, cols = 4, 3, 5
    M = synth.random_uints((rows, cols), w, 5, "M")
    v = synth.random_uints(cols, w, 5, "v")
    dM, oM = E.enc_ints(M, w, 6, "M")
    dv, ov = E.enc_ints(v, w, 6, "v")
    y = E.out((rows, w))
    E.ctx.matvec(w, dM, dv, y)
    want, _ = E.orc.matvec(E.P, E.obk, E.oksk, w, oM, ov)
    got = E.host(y)
    assert np.array_equal(got, want)
    assert np.array_equal(E.dec_ints(got), (M * v[None, :]).sum(axis=1) % (1 << w))


def test_mixed_jobs_and_schedules_agree(small):
    """Jobs of uneven depth share one level schedule; the result of every job
    equals its oracle result, and equals the result of the same job run
    alone, with graphs off, and gate by gate (one launch pair per gate)."""
    E = small
    api = E.api
    a8, b8 = synth.int_pairs(2, 8, 7, "x8")
    a4, b4 = synth.int_pairs(3, 4, 7, "x4")
    ga, gb = synth.random_bits(5, 7, "ga"), synth.random_bits(5, 7, "gb")
    d8a, o8a = E.enc_ints(a8, 8, 8, "x8a")
    d8b, o8b = E.enc_ints(b8, 8, 8, "x8b")
    d4a, o4a = E.enc_ints(a4, 4, 8, "x4a")
    d4b, o4b = E.enc_ints(b4, 4, 8, "x4b")
    dga, oga = E.enc_ints(ga, 1, 8, "ga")
    dgb, ogb = E.enc_ints(gb, 1, 8, "gb")

    def run(mode):
        outs = [E.out((2, 8)), E.out((3, 4)), E.out((5, 1))]
        jobs = [dict(kind=api.ADD, width=8, batch=2, in0=d8a, in1=d8b, out=outs[0]),
                dict(kind=api.MUL, width=4, batch=3, in0=d4a, in1=d4b, out=outs[1]),
                dict(kind=api.GATE, width=api.XOR, batch=5, in0=dga, in1=dgb, out=outs[2])]
        if mode == "alone":
            for j in jobs:
                E.ctx.run_jobs([j])
        else:
            E.ctx.set_option(api.OPT_GRAPHS, mode != "nograph")
            E.ctx.set_option(api.OPT_PER_GATE, mode == "pergate")
            E.ctx.set_option(api.OPT_SCHEDULE, api.SCHED_ASAP if mode == "asap" else
                             api.SCHED_BALANCED)
            E.ctx.set_option(api.OPT_LEVEL_WIDTH, 7 if mode == "narrow" else 0)
            E.ctx.run_jobs(jobs)
            E.ctx.set_option(api.OPT_GRAPHS, 1)
            E.ctx.set_option(api.OPT_PER_GATE, 0)
            E.ctx.set_option(api.OPT_SCHEDULE, api.SCHED_BALANCED)
            E.ctx.set_option(api.OPT_LEVEL_WIDTH, 0)
        return [E.host(o) for o in outs]

    mixed = run("graph")
    want_add, _ = E.orc.add(E.P, E.obk, E.oksk, 8, o8a, o8b)
    want_mul, _ = E.orc.mul(E.P, E.obk, E.oksk, 4, o4a, o4b)
    want_xor = E.orc.gates(E.P, E.obk, E.oksk, np.full(5, 3, np.uint8), oga[:, 0], ogb[:, 0])
    assert np.array_equal(mixed[0], want_add)
    assert np.array_equal(mixed[1], want_mul)
    assert np.array_equal(mixed[2][:, 0], want_xor)
    for mode in ("alone", "nograph", "pergate", "asap", "narrow"):
        other = run(mode)
        for x, y in zip(mixed, other):
            assert np.array_equal(x, y), mode


# ----------------------------------------------------------- full size, n = 500

@pytest.fixture(scope="module")
def full(orc):
    e = Env(orc, 500, synth.MASTER_SEED)
    # the launch configuration the benchmark times: tuned CTA shapes and
    # key-switch kernels, and the wave size each schedule picks from them
    e.ctx.autotune()
    yield e
    e.ctx.close()


def test_config1_add32_x256(full):
    """256 32-bit additions (39,424 bootstraps, depth 62): every sum decrypts
    correctly; sampled bit-0 outputs (one XOR of fresh inputs) are bit-exact."""
    E = full
    a, b = synth.int_pairs(256, 32, synth.MASTER_SEED + 1, "add32")
    da, oa = E.enc_ints(a, 32, synth.MASTER_SEED + 1, "add32a")
    db, ob = E.enc_ints(b, 32, synth.MASTER_SEED + 1, "add32b")
    R = E.out((256, 32))
    E.ctx.add_n(32, da, db, R)
    got = E.host(R)
    assert np.array_equal(E.dec_ints(got), (a + b) % (1 << 32))
    idx = np.array([0, 77, 255])
    want = E.orc.gates(E.P, E.obk, E.oksk, np.full(3, 3, np.uint8), oa[idx, 0], ob[idx, 0])
    assert np.array_equal(got[idx, 0], want)
    assert E.ctx.status() == 0


def test_config1_sampled_instances_bit_exact(full):
    """The bench workload at full parameters (n = 500) and in its launch
    configuration (one 256-instance schedule, tuned shapes): 16 sampled
    32-bit additions are recomputed by the oracle gate by gate (154
    bootstraps each, 62 levels deep) and all 32 output ciphertexts of each
    are bit-exact."""
    E = full
    a, b = synth.int_pairs(256, 32, synth.MASTER_SEED + 1, "add32")
    da, oa = E.enc_ints(a, 32, synth.MASTER_SEED + 1, "add32a")
    db, ob = E.enc_ints(b, 32, synth.MASTER_SEED + 1, "add32b")
    R = E.out((256, 32))
    E.ctx.add_n(32, da, db, R)
    got = E.host(R)
    idx = np.array([0, 1, 17, 40, 63, 64, 99, 127, 128, 150, 191, 200, 222, 240, 254, 255])
    want, gates = E.orc.add(E.P, E.obk, E.oksk, 32, np.ascontiguousarray(oa[idx]),
                            np.ascontiguousarray(ob[idx]))
    assert gates == len(idx) * 154
    assert np.array_equal(got[idx], want)
    assert E.ctx.status() == 0


def test_shallow_circuits_full_parameters_decrypt(full):
    """The low-depth circuits at n = 500: 256 parallel-prefix additions and
    64 Dadda multiplications of 32 bits (197K bootstraps, mostly majority
    gates) in one schedule; every output decrypts to the integer result.
    Bit-exact parity at n = 16 cannot see the noise, so this checks that
    every gate of these circuits keeps its decision margin."""
    E = full
    api = E.api
    a, b = synth.int_pairs(256, 32, 81, "px")
    c, d = synth.int_pairs(64, 32, 82, "dd")
    da, _ = E.enc_ints(a, 32, 81, "pxa")
    db, _ = E.enc_ints(b, 32, 81, "pxb")
    dc, _ = E.enc_ints(c, 32, 82, "dda")
    dd, _ = E.enc_ints(d, 32, 82, "ddb")
    R1, R2 = E.out((256, 32)), E.out((64, 32))
    E.ctx.run_jobs([dict(kind=api.ADD_PREFIX, width=32, batch=256, in0=da, in1=db, out=R1),
                    dict(kind=api.MUL_DADDA, width=32, batch=64, in0=dc, in1=dd, out=R2)])
    assert np.array_equal(E.dec_ints(E.host(R1)), (a + b) % (1 << 32))
    assert np.array_equal(E.dec_ints(E.host(R2)), (c * d) % (1 << 32))
    assert E.ctx.status() == 0


def test_lone_request_schedules_agree(full):
    """One 32-bit multiplication alone (sequential and Dadda) at n = 500 in
    the tuned configuration, where the schedule may round levels to one
    bootstrap per SM for latency, and again with levels forced to waves of
    608 gates: the ciphertexts are identical word for word and decrypt to
    the product."""
    E = full
    api = E.api
    a, b = synth.int_pairs(1, 32, 91, "lone")
    da, _ = E.enc_ints(a, 32, 91, "lonea")
    db, _ = E.enc_ints(b, 32, 91, "loneb")
    for kind in (api.MUL_DADDA, api.MUL):
        R1, R2 = E.out((1, 32)), E.out((1, 32))
        E.ctx.run_jobs([dict(kind=kind, width=32, batch=1, in0=da, in1=db, out=R1)])
        E.ctx.set_option(api.OPT_LEVEL_WIDTH, 608)
        try:
            E.ctx.run_jobs([dict(kind=kind, width=32, batch=1, in0=da, in1=db, out=R2)])
        finally:
            E.ctx.set_option(api.OPT_LEVEL_WIDTH, 0)
        g1, g2 = E.host(R1), E.host(R2)
        assert np.array_equal(g1, g2)
        assert np.array_equal(E.dec_ints(g1), (a * b) % (1 << 32))
    assert E.ctx.status() == 0


def test_config2_mul16_mul32_mixed(full):
    """64 16-bit and 64 32-bit multiplications in one schedule (222,208
    bootstraps, uneven depths 56 and 120), n = 500: every product decrypts
    correctly, and one 16-bit and one 32-bit instance are recomputed by the
    oracle gate by gate (648 + 2,824 bootstraps, 120 levels deep) with every
    output ciphertext bit-exact."""
    E = full
    api = E.api
    a16, b16 = synth.int_pairs(64, 16, synth.MASTER_SEED + 2, "mul16")
    a32, b32 = synth.int_pairs(64, 32, synth.MASTER_SEED + 2, "mul32")
    d16a, o16a = E.enc_ints(a16, 16, synth.MASTER_SEED + 2, "m16a")
    d16b, o16b = E.enc_ints(b16, 16, synth.MASTER_SEED + 2, "m16b")
    d32a, o32a = E.enc_ints(a32, 32, synth.MASTER_SEED + 2, "m32a")
    d32b, o32b = E.enc_ints(b32, 32, synth.MASTER_SEED + 2, "m32b")
    R16, R32 = E.out((64, 16)), E.out((64, 32))
    E.ctx.run_jobs([dict(kind=api.MUL, width=16, batch=64, in0=d16a, in1=d16b, out=R16),
                    dict(kind=api.MUL, width=32, batch=64, in0=d32a, in1=d32b, out=R32)])
    g16, g32 = E.host(R16), E.host(R32)
    assert E.ctx.status() == 0
    assert np.array_equal(E.dec_ints(g16), (a16 * b16) % (1 << 16))
    assert np.array_equal(E.dec_ints(g32), (a32 * b32) % (1 << 32))
    i16, i32 = 9, 41
    want16, n16 = E.orc.mul(E.P, E.obk, E.oksk, 16, o16a[[i16]], o16b[[i16]])
    want32, n32 = E.orc.mul(E.P, E.obk, E.oksk, 32, o32a[[i32]], o32b[[i32]])
    assert (n16, n32) == (648, 2824)
    assert np.array_equal(g16[i16], want16[0])
    assert np.array_equal(g32[i32], want32[0])


def test_config3_matvec16(full):
    """16x16 matrix times 16-vector, 16-bit (183,648 bootstraps), n = 500:
    every output decrypts correctly, and one full output row (16 products
    and the adder tree, 11,478 bootstraps) is recomputed by the oracle gate
    by gate with all 16 output ciphertexts bit-exact."""
    E = full
    M = synth.random_uints((16, 16), 16, synth.MASTER_SEED + 3, "M")
    v = synth.random_uints(16, 16, synth.MASTER_SEED + 3, "v")
    dM, oM = E.enc_ints(M, 16, synth.MASTER_SEED + 3, "M")
    dv, ov = E.enc_ints(v, 16, synth.MASTER_SEED + 3, "v")
    y = E.out((16, 16))
    E.ctx.matvec(16, dM, dv, y)
    got = E.host(y)
    assert E.ctx.status() == 0
    assert np.array_equal(E.dec_ints(got), (M * v[None, :]).sum(axis=1) % (1 << 16))
    r = 6
    want, gates = E.orc.matvec(E.P, E.obk, E.oksk, 16, np.ascontiguousarray(oM[[r]]), ov)
    assert gates == 16 * 648 + 15 * 74
    assert np.array_equal(got[r], want[0])


@pytest.mark.parametrize("kind_name,w", [("ADD_MAJ", 32), ("ADD_NW", 8), ("MUL_TREE", 8),
                                         ("ADD_MAJ", 1), ("MUL_TREE", 3), ("MUL_TREE_MAJ", 8),
                                         ("MUL_TREE_MAJ", 5), ("ADD_PREFIX", 32), ("ADD_PREFIX", 6),
                                         ("MUL_DADDA", 8), ("MUL_DADDA", 6)])
def test_next_circuits_bit_exact(small, kind_name, w):
    """Majority-carry adder (3-input MAJ gates), the paper's number-wise
    adder, tree-accumulated multiplication (ripple or majority carries), the
    parallel-prefix adder (majority gates) and the Dadda multiplier,
    bit-exact against the oracle."""
    E = small
    api = E.api
    kind = getattr(api, kind_name)
    a, b = synth.int_pairs(2, w, 11, f"{kind_name}{w}")
    da, oa = E.enc_ints(a, w, 12, f"na{kind_name}{w}")
    db, ob = E.enc_ints(b, w, 12, f"nb{kind_name}{w}")
    R = E.out((2, w))
    E.ctx.run_jobs([dict(kind=kind, width=w, batch=2, in0=da, in1=db, out=R)])
    fn = {"ADD_MAJ": E.orc.add_maj, "ADD_NW": E.orc.add_nw, "MUL_TREE": E.orc.mul_tree,
          "MUL_TREE_MAJ": E.orc.mul_tree_maj, "ADD_PREFIX": E.orc.add_prefix,
          "MUL_DADDA": E.orc.mul_dadda}[kind_name]
    want, g = fn(E.P, E.obk, E.oksk, w, oa, ob)
    got = E.host(R)
    assert np.array_equal(got, want)
    assert g == 2 * api.circuit_info(kind, w)[0]
    assert E.ctx.status() == 0


def test_majority_adder_in_serving_and_mixed(small):
    """3-input gates through the serving loop and in a mixed schedule."""
    E = small
    api = E.api
    a, b = synth.int_pairs(1, 16, 13, "sm16")
    da, oa = E.enc_ints(a, 16, 14, "sma")
    db, ob = E.enc_ints(b, 16, 14, "smb")
    want, _ = E.orc.add_maj(E.P, E.obk, E.oksk, 16, oa, ob)
    R1, R2, R3 = E.out((1, 16)), E.out((1, 16)), E.out((1, 16))
    E.ctx.run_jobs([dict(kind=api.ADD_MAJ, width=16, batch=1, in0=da, in1=db, out=R1),
                    dict(kind=api.ADD, width=16, batch=1, in0=da, in1=db, out=R2)])
    kd, dv = E.kd, api.to_device
    bk, ksk = api.keygen(E.p, dv(kd.s), dv(kd.S), dv(kd.bk_mask), dv(kd.bk_noise),
                         dv(kd.ksk_mask), dv(kd.ksk_noise))
    ctx = api.Context(E.p)
    ctx.set_keys(bk, ksk)
    ctx.serve_start(64 << 20)
    rid = ctx.serve_submit(api.ADD_MAJ, 16, da[0], db[0], R3[0])
    ctx.serve_wait(rid, 60000)
    ctx.serve_stop()
    ctx.close()
    assert np.array_equal(E.host(R1), want)
    assert np.array_equal(E.host(R3), want)
    assert np.array_equal(E.dec_ints(E.host(R2)), (a + b) % (1 << 16))


@pytest.mark.parametrize("kind_name,w", [("MUL_FULL", 2), ("MUL_FULL", 8), ("MUL_KARATSUBA", 9),
                                         ("MUL_KARATSUBA", 16), ("MUL_KARATSUBA", 32)])
def test_full_products_bit_exact(small, kind_name, w):
    """Full products (2w output rows): the naive product and Karatsuba
    (Algorithm "karatsuba", vector form of section V-B), bit-exact against
    the oracle, with all-ones operands among the instances."""
    E = small
    api = E.api
    kind = getattr(api, kind_name)
    a, b = synth.int_pairs(2, w, 13, f"{kind_name}{w}")
    a[0] = b[0] = (1 << w) - 1
    da, oa = E.enc_ints(a, w, 14, f"fa{kind_name}{w}")
    db, ob = E.enc_ints(b, w, 14, f"fb{kind_name}{w}")
    R = E.out((2, 2 * w))
    E.ctx.run_jobs([dict(kind=kind, width=w, batch=2, in0=da, in1=db, out=R)])
    fn = E.orc.mul_full if kind_name == "MUL_FULL" else E.orc.mul_karatsuba
    want, g = fn(E.P, E.obk, E.oksk, w, oa, ob)
    got = E.host(R)
    assert np.array_equal(got, want)
    assert g == 2 * api.circuit_info(kind, w)[0]
    bits = E.orc.decrypt_bits(E.P, E.kd.s, got)
    assert [sum(int(v) << i for i, v in enumerate(r)) for r in bits] == \
        [int(x) * int(y) for x, y in zip(a, b)]
    assert E.ctx.status() == 0


def test_full_product_width_checked(small):
    """w = 1 has a constant top product bit and is refused; so is w > 64."""
    E = small
    api = E.api
    R = E.out((1, 2))
    A = E.out((1, 1))
    for w in (1, 65):
        with pytest.raises(RuntimeError):
            E.ctx.run_jobs([dict(kind=api.MUL_KARATSUBA, width=w, batch=1, in0=A, in1=A, out=R)])
    assert E.ctx.status() == 0
