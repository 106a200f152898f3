"""Edge cases of the C ABI on the GPU: empty batches, opcodes without their
inputs, parameter sets outside the supported range, trivial (zero-mask)
ciphertexts for which every CMux is skipped, the largest LWE dimension
(n = 511) bit-exact against the oracle, and a 100,000-gate batch checked
by decryption on every output and by the oracle on a sample, and a key
switch over more tiles than one launch grid holds."""
import numpy as np
import pytest

from conftest import oparams
from paper_2005_01945_gb300 import synth

pytestmark = pytest.mark.gpu
MU = 1 << 29


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


class Env:
    def __init__(self, orc, n, seed):
        import torch
        from paper_2005_01945_gb300 import api, build
        build.build()
        self.torch, self.api, self.orc = torch, api, orc
        self.p = synth.TFHEParams(n=n)
        self.P = oparams(self.p)
        self.kd = kd = synth.key_draws(self.p, seed)
        d = api.to_device
        self.bk, self.ksk = api.keygen(self.p, d(kd.s), d(kd.S), d(kd.bk_mask), d(kd.bk_noise),
                                       d(kd.ksk_mask), d(kd.ksk_noise))
        self.ctx = api.Context(self.p)
        self.ctx.set_keys(self.bk, self.ksk)
        self.s_dev = d(kd.s)
        self.obk = orc.keygen_bk(self.P, kd.s, kd.S, kd.bk_mask, kd.bk_noise)
        self.oksk = orc.keygen_ksk(self.P, kd.s, kd.S, kd.ksk_mask, kd.ksk_noise)

    def fresh(self, count, seed, tag):
        bits = synth.random_bits((2, count), seed, tag)
        cd = synth.ct_draws(self.p, (2, count), seed, tag)
        cts = self.orc.encrypt_bits(self.P, self.kd.s, cd.mask, cd.noise, bits)
        d = self.api.to_device
        dev = self.api.encrypt_bits(self.p, self.s_dev, d(cd.mask), d(cd.noise), d(bits))
        return bits, cts, dev

    def out(self, count):
        return self.torch.full((count, 512), 7, dtype=self.torch.int32, device="cuda")


@pytest.fixture(scope="module")
def env(orc):
    e = Env(orc, 500, synth.MASTER_SEED + 21)
    yield e
    e.ctx.close()


def test_empty_batches_are_no_ops(env):
    """Zero gates, zero key switches and zero-instance circuits return OK and
    write nothing."""
    torch, api, ctx = env.torch, env.api, env.ctx
    ops = torch.empty(0, dtype=torch.uint8, device="cuda")
    a = torch.empty((0, 512), dtype=torch.int32, device="cuda")
    out = env.out(4)
    before = out.clone()
    ctx.bootstrap_gates(ops, a, a, out[:0])
    ctx.keyswitch(torch.empty((0, api.BIG_STRIDE), dtype=torch.int32, device="cuda"), out[:0])
    A = torch.empty((0, 8, 512), dtype=torch.int32, device="cuda")
    ctx.run_jobs([dict(kind=api.ADD, width=8, batch=0, in0=A, in1=A, out=A)])
    torch.cuda.synchronize()
    assert torch.equal(out, before)
    assert ctx.status() == 0


@pytest.mark.parametrize("bad", [6, 11, 200])
def test_opcode_without_inputs_is_flagged(env, bad):
    """A 3-input MAJ or an unknown opcode in tfhe_bootstrap_gates sets bit 3
    of the status word and yields the all-zero row; the other gates of the
    batch stay bit-exact."""
    api, orc = env.api, env.orc
    count = 5
    bits, cts, dev = env.fresh(count, 3, f"bad{bad}")
    ops = np.array([1, bad, 3, 0, 5], dtype=np.uint8)
    out = env.out(count)
    env.ctx.bootstrap_gates(api.to_device(ops), dev[0], dev[1], out)
    assert env.ctx.status() == 8
    got = _u32(out)
    good = np.array([0, 2, 3, 4])
    want = orc.gates(env.P, env.obk, env.oksk, ops[good], cts[0][good], cts[1][good])
    assert np.array_equal(got[good, :env.p.n + 1], want)
    assert not got[1].any()
    assert env.ctx.status() == 0     # reading the word clears it


def test_unsupported_parameters_rejected(env):
    """n above 511 or a ring other than N = 1024 is refused at creation."""
    api = env.api
    for kw in (dict(n=512), dict(N=2048), dict(l=3), dict(bg_bit=8)):
        with pytest.raises(api.TFHEError):
            api.Context(synth.TFHEParams(**kw))


def test_trivial_ciphertexts_skip_every_cmux(env):
    """Zero-mask samples (0, +-1/8) mod-switch every a_i to 0, so every CMux
    is skipped; the result is the rotated test vector, key-switched, equal to
    the oracle's."""
    torch, api, orc, p = env.torch, env.api, env.orc, env.p
    count = 6
    rows = np.zeros((2, count, p.n + 1), dtype=np.uint32)
    rows[:, :, p.n] = np.where(synth.random_bits((2, count), 5, "triv"), MU, (1 << 32) - MU)
    dev = torch.zeros((2, count, 512), dtype=torch.int32, device="cuda")
    dev[:, :, :p.n + 1] = torch.from_numpy(rows.view(np.int32)).cuda()
    ops = np.array([0, 1, 2, 3, 4, 5], dtype=np.uint8)
    out = env.out(count)
    env.ctx.bootstrap_gates(api.to_device(ops), dev[0], dev[1], out)
    want = orc.gates(env.P, env.obk, env.oksk, ops, rows[0], rows[1])
    assert np.array_equal(_u32(out)[:, :p.n + 1], want)
    assert env.ctx.status() == 0


def test_largest_lwe_dimension_bit_exact(orc):
    """n = 511, the largest LWE dimension the row stride holds (n + 1 = 512
    words, no padding left), bit-exact against the oracle."""
    e = Env(orc, 511, synth.MASTER_SEED + 22)
    try:
        count = 6
        bits, cts, dev = e.fresh(count, 9, "n511")
        ops = np.array([0, 1, 2, 3, 4, 5], dtype=np.uint8)
        out = e.out(count)
        e.ctx.bootstrap_gates(e.api.to_device(ops), dev[0], dev[1], out)
        want = orc.gates(e.P, e.obk, e.oksk, ops, cts[0], cts[1])
        assert np.array_equal(_u32(out), want)
        assert e.ctx.status() == 0
    finally:
        e.ctx.close()


def test_hundred_thousand_gates(env):
    """100,000 gates in one call (one blind-rotation launch whose persistent
    CTAs loop over about 165 waves of 608 bootstraps, and one key-switch
    launch): every output decrypts to its truth-table value, and 8 sampled
    outputs equal the oracle's."""
    api, orc, p = env.api, env.orc, env.p
    count = 100_000
    bits, cts, dev = env.fresh(count, 13, "big")
    ops = (np.arange(count) * 7 % 6).astype(np.uint8)
    out = env.out(count)
    env.ctx.bootstrap_gates(api.to_device(ops), dev[0], dev[1], out)
    got = _u32(out)
    dec = orc.decrypt_bits(env.P, env.kd.s, got[:, :p.n + 1])
    a, b = bits[0].astype(bool), bits[1].astype(bool)
    table = [~(a & b), a & b, a | b, a ^ b, ~(a | b), ~(a ^ b)]
    truth = np.choose(ops, table)
    assert np.array_equal(dec.astype(bool), truth)
    sample = synth._gen(41, "big-sample").choice(count, 8, replace=False)
    want = orc.gates(env.P, env.obk, env.oksk, ops[sample], cts[0][sample], cts[1][sample])
    assert np.array_equal(got[sample, :p.n + 1], want)
    assert env.ctx.status() == 0


def test_keyswitch_beyond_one_grid_of_tiles(env):
    """4,194,310 LWE_N samples: 65,537 tiles of 64 gates, more than the
    65,535 that one launch grid holds, so the tiled key switch's CTAs loop
    over a second tile.  Rows around both grid boundaries (and the last,
    ragged tile) are bit-exact against the oracle."""
    torch, api, orc, p = env.torch, env.api, env.orc, env.p
    count = 65535 * 64 + 70
    gen = torch.Generator(device="cuda").manual_seed(17)
    big = torch.randint(-2**31, 2**31 - 1, (count, api.BIG_STRIDE), dtype=torch.int32,
                        device="cuda", generator=gen)
    out = torch.empty((count, 512), dtype=torch.int32, device="cuda")
    env.ctx.set_option(api.OPT_KS_KERNEL, api.KS_TILED)
    try:
        env.ctx.keyswitch(big, out)
    finally:
        env.ctx.set_option(api.OPT_KS_KERNEL, 0)
    edge = 65535 * 64
    sample = np.array([0, 63, 64, edge - 1, edge, edge + 63, edge + 64, count - 1])
    idx = torch.from_numpy(sample).cuda()
    rows = big.index_select(0, idx).cpu().numpy().view(np.uint32)
    got = out.index_select(0, idx).cpu().numpy().view(np.uint32)
    del big, out
    want = orc.keyswitch(env.P, env.oksk, np.ascontiguousarray(rows[:, :p.N + 1]))
    assert np.array_equal(got[:, :p.n + 1], want)
    assert not got[:, p.n + 1:].any()
    assert env.ctx.status() == 0


def test_keyswitch_wait_timeout_is_reported_and_recoverable(env):
    """Failure detection without a GPU fault: with the stall test hook every
    stage of the tiled key switch also waits on an mbarrier that nothing
    completes.  Each bounded wait runs out, the kernel records the timeout
    (status bit 2), lets the copies it issued land, and returns; the next call on the same context,
    hook off, is bit-exact against the oracle."""
    torch, api, orc, p = env.torch, env.api, env.orc, env.p
    count = 70
    rng = np.random.default_rng(23)
    big = rng.integers(0, 1 << 32, size=(count, api.BIG_STRIDE), dtype=np.uint64)
    big = big.astype(np.uint32)
    dbig = api.to_device(big)
    out = torch.zeros((count, 512), dtype=torch.int32, device="cuda")
    env.ctx.set_option(api.OPT_KS_KERNEL, api.KS_TILED)
    try:
        env.ctx.set_option(api.OPT_TEST_KS_STALL, 1)
        try:
            env.ctx.keyswitch(dbig, out)
        finally:
            env.ctx.set_option(api.OPT_TEST_KS_STALL, 0)
        assert env.ctx.status() == 4
        env.ctx.keyswitch(dbig, out)
    finally:
        env.ctx.set_option(api.OPT_KS_KERNEL, 0)
    want = orc.keyswitch(env.P, env.oksk, np.ascontiguousarray(big[:, :p.N + 1]))
    assert np.array_equal(_u32(out)[:, :p.n + 1], want)
    assert env.ctx.status() == 0
