"""GPU parity of gate bootstrapping through the C ABI, bit-exact against the
oracle: client key generation and encryption, the blind-rotation +
extraction stage, the key-switch stage, and whole gates."""
import numpy as np
import pytest

from conftest import center, oparams, trivial_rotation
from paper_2005_01945_gb300 import synth

pytestmark = pytest.mark.gpu
M32 = 1 << 32
MU = 1 << 29


@pytest.fixture(scope="module")
def gpu(orc):
    import torch
    from paper_2005_01945_gb300 import api, build
    build.build()
    p = synth.TFHEParams()
    P = oparams(p)
    kd = synth.key_draws(p, synth.MASTER_SEED)
    d = api.to_device
    bk, ksk = api.keygen(p, d(kd.s), d(kd.S), d(kd.bk_mask), d(kd.bk_noise), d(kd.ksk_mask),
                         d(kd.ksk_noise))
    ctx = api.Context(p)
    ctx.set_keys(bk, ksk)
    obk = orc.keygen_bk(P, kd.s, kd.S, kd.bk_mask, kd.bk_noise)
    oksk = orc.keygen_ksk(P, kd.s, kd.S, kd.ksk_mask, kd.ksk_noise)
    torch.cuda.synchronize()
    yield dict(torch=torch, api=api, p=p, P=P, kd=kd, ctx=ctx, bk=bk, ksk=ksk, obk=obk,
               oksk=oksk, s_dev=d(kd.s))
    ctx.close()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def test_keygen_bit_exact(gpu):
    assert np.array_equal(_u32(gpu["bk"]), gpu["obk"])
    assert np.array_equal(_u32(gpu["ksk"]), gpu["oksk"])


def test_encrypt_and_phase_bit_exact(gpu, orc):
    api, p, P, kd = gpu["api"], gpu["p"], gpu["P"], gpu["kd"]
    bits = synth.random_bits(777, 3, "enc")
    cd = synth.ct_draws(p, 777, 3, "enc")
    ct = api.encrypt_bits(p, gpu["s_dev"], api.to_device(cd.mask), api.to_device(cd.noise),
                          api.to_device(bits))
    oct_ = orc.encrypt_bits(P, kd.s, cd.mask, cd.noise, bits)
    got = _u32(ct)
    assert np.array_equal(got[:, :p.n + 1], oct_)
    assert not got[:, p.n + 1:].any()
    ph = _u32(api.phase(p, gpu["s_dev"], ct))
    assert np.array_equal(ph, orc.phase(P, kd.s, oct_))


def _fresh(gpu, orc, count, seed, tag, zero_some=False):
    """count ciphertext pairs: device tensors and oracle arrays of the same draws."""
    api, p, P, kd = gpu["api"], gpu["p"], gpu["P"], gpu["kd"]
    bits = synth.random_bits((2, count), seed, tag)
    cd = synth.ct_draws(p, (2, count), seed, tag)
    if zero_some:   # mask words that mod-switch to 0 exercise the skipped CMux
        cd.mask[:, :, ::7] = 0
    cts = orc.encrypt_bits(P, kd.s, cd.mask, cd.noise, bits)
    dev = api.encrypt_bits(p, gpu["s_dev"], api.to_device(cd.mask), api.to_device(cd.noise),
                           api.to_device(bits))
    return bits, cts, dev


@pytest.mark.parametrize("count", [1, 8, 37])
def test_gates_bit_exact(gpu, orc, count):
    torch, api, p, P, kd = gpu["torch"], gpu["api"], gpu["p"], gpu["P"], gpu["kd"]
    bits, cts, dev = _fresh(gpu, orc, count, 10 + count, f"g{count}", zero_some=count == 37)
    ops = (np.arange(count) % 6).astype(np.uint8)
    out = torch.zeros((count, 512), dtype=torch.int32, device="cuda")
    gpu["ctx"].bootstrap_gates(api.to_device(ops), dev[0], dev[1], out)
    want = orc.gates(P, gpu["obk"], gpu["oksk"], ops, cts[0], cts[1])
    got = _u32(out)
    assert np.array_equal(got[:, :p.n + 1], want)
    assert not got[:, p.n + 1:].any()
    assert gpu["ctx"].status() == 0


def test_config0_gates8(gpu, orc):
    """Config 0: NAND, NAND, AND, AND, OR, OR, XOR, XOR on 16 fresh encryptions."""
    torch, api, p, P, kd = gpu["torch"], gpu["api"], gpu["p"], gpu["P"], gpu["kd"]
    ops, ba, bb = synth.gates8_inputs(synth.MASTER_SEED)
    cd = synth.ct_draws(p, (2, 8), synth.MASTER_SEED, "gates8")
    ca = orc.encrypt_bits(P, kd.s, cd.mask[0], cd.noise[0], ba)
    cb = orc.encrypt_bits(P, kd.s, cd.mask[1], cd.noise[1], bb)
    da = api.encrypt_bits(p, gpu["s_dev"], api.to_device(cd.mask[0]), api.to_device(cd.noise[0]),
                          api.to_device(ba))
    db = api.encrypt_bits(p, gpu["s_dev"], api.to_device(cd.mask[1]), api.to_device(cd.noise[1]),
                          api.to_device(bb))
    out = torch.empty((8, 512), dtype=torch.int32, device="cuda")
    gpu["ctx"].bootstrap_gates(api.to_device(ops), da, db, out)
    want = orc.gates(P, gpu["obk"], gpu["oksk"], ops, ca, cb)
    assert np.array_equal(_u32(out)[:, :p.n + 1], want)
    truth = {0: lambda a, b: 1 - (a & b), 1: lambda a, b: a & b, 2: lambda a, b: a | b,
             3: lambda a, b: a ^ b}
    dec = orc.decrypt_bits(P, kd.s, want)
    assert all(dec[k] == truth[int(ops[k])](int(ba[k]), int(bb[k])) for k in range(8))


def test_blind_rotate_extract_stage(gpu, orc):
    torch, api, p, P, kd = gpu["torch"], gpu["api"], gpu["p"], gpu["P"], gpu["kd"]
    count = 6
    bits, cts, dev = _fresh(gpu, orc, count, 20, "br", zero_some=True)
    big = torch.zeros((count, 1056), dtype=torch.int32, device="cuda")
    gpu["ctx"].blind_rotate_extract(None, dev[0], None, big)
    abar = orc.modswitch(cts[0].reshape(-1), p.N).reshape(count, p.n + 1)
    acc = orc.blind_rotate(P, gpu["obk"], abar)
    want = np.stack([orc.sample_extract(P, acc[g]) for g in range(count)])
    assert np.array_equal(_u32(big)[:, :p.N + 1], want)


@pytest.mark.parametrize("count", [3, 5000])
def test_keyswitch_stage(gpu, orc, count):
    """The default key switch (tiled kernel): a small batch splits j over
    many CTAs (reductions into the output), a large one stores directly."""
    torch, api, p, P = gpu["torch"], gpu["api"], gpu["p"], gpu["P"]
    rng = np.random.default_rng(count)
    big = rng.integers(0, M32, size=(count, 1056), dtype=np.uint64).astype(np.uint32)
    out = torch.zeros((count, 512), dtype=torch.int32, device="cuda")
    gpu["ctx"].keyswitch(api.to_device(big), out)
    sample = np.arange(count) if count < 100 else rng.choice(count, 64, replace=False)
    want = orc.keyswitch(P, gpu["oksk"], np.ascontiguousarray(big[sample, :p.N + 1]))
    got = _u32(out)[sample]
    assert np.array_equal(got[:, :p.n + 1], want)
    assert not got[:, p.n + 1:].any()


@pytest.mark.parametrize("kernel,count", [(64, 1), (64, 63), (64, 65), (64, 700), (64, 5000),
                                          (1, 40), (4, 40), (32, 300)])
def test_keyswitch_kernels_bit_exact(gpu, orc, kernel, count):
    """Each key-switch kernel on uniform LWE_N samples: the tiled kernel
    (64 gates per CTA, key rows staged in shared memory) on one gate, a
    ragged tile, two tiles, a j-split over 11 tiles (reductions into the
    output) and 79 tiles (direct stores, no split); the direct kernel with
    1, 4 and 32 j-chunks.  Sampled rows (and the first and last) are
    bit-exact against the oracle; padding words stay zero."""
    torch, api, p, P = gpu["torch"], gpu["api"], gpu["p"], gpu["P"]
    rng = np.random.default_rng(1000 + count + kernel)
    big = rng.integers(0, M32, size=(count, 1056), dtype=np.uint64).astype(np.uint32)
    out = torch.full((count, 512), -1, dtype=torch.int32, device="cuda")
    gpu["ctx"].set_option(api.OPT_KS_KERNEL, kernel)
    try:
        gpu["ctx"].keyswitch(api.to_device(big), out)
    finally:
        gpu["ctx"].set_option(api.OPT_KS_KERNEL, 0)
    if count <= 70:
        sample = np.arange(count)
    else:
        sample = np.unique(np.concatenate([[0, count - 1],
                                           rng.choice(count, 40, replace=False)]))
    want = orc.keyswitch(P, gpu["oksk"], np.ascontiguousarray(big[sample, :p.N + 1]))
    got = _u32(out)[sample]
    assert np.array_equal(got[:, :p.n + 1], want)
    assert not got[:, p.n + 1:].any()
    assert gpu["ctx"].status() == 0


def test_keyswitch_kernels_agree_on_gates(gpu, orc):
    """Whole gates (blind rotation + key switch) with the tiled key switch
    and with the direct one give identical ciphertexts."""
    torch, api = gpu["torch"], gpu["api"]
    count = 300
    bits, cts, dev = _fresh(gpu, orc, count, 55, "ksk2")
    ops = (np.arange(count) % 6).astype(np.uint8)
    outs = []
    for kernel in (api.KS_TILED, 8):
        out = torch.zeros((count, 512), dtype=torch.int32, device="cuda")
        gpu["ctx"].set_option(api.OPT_KS_KERNEL, kernel)
        try:
            gpu["ctx"].bootstrap_gates(api.to_device(ops), dev[0], dev[1], out)
        finally:
            gpu["ctx"].set_option(api.OPT_KS_KERNEL, 0)
        outs.append(out)
    assert torch.equal(outs[0], outs[1])


def test_keys_save_and_load(gpu, orc, tmp_path):
    """Checkpoint / resume of the device keys: a new context loads the file
    the first one saved and gives the same gates (bit-exact against the
    oracle); a flipped payload byte, keys of other parameters and a missing
    file are refused with TFHE_EINVAL."""
    torch, api, p, P = gpu["torch"], gpu["api"], gpu["p"], gpu["P"]
    path = tmp_path / "keys.tfhegb"
    gpu["ctx"].save_keys(path)
    count = 9
    bits, cts, dev = _fresh(gpu, orc, count, 88, "keyio")
    ops = (np.arange(count) % 6).astype(np.uint8)
    ctx2 = api.Context(p)
    try:
        ctx2.load_keys(path)
        outs = []
        for ctx in (gpu["ctx"], ctx2):
            out = torch.zeros((count, 512), dtype=torch.int32, device="cuda")
            ctx.bootstrap_gates(api.to_device(ops), dev[0], dev[1], out)
            outs.append(out)
        assert torch.equal(outs[0], outs[1])
        want = orc.gates(P, gpu["obk"], gpu["oksk"], ops, cts[0], cts[1])
        assert np.array_equal(_u32(outs[1])[:, :p.n + 1], want)
        bad = tmp_path / "bad.tfhegb"
        raw = bytearray(path.read_bytes())
        raw[len(raw) // 2] ^= 1
        bad.write_bytes(bytes(raw))
        with pytest.raises(api.TFHEError) as err:
            ctx2.load_keys(bad)
        assert err.value.code == -1
        with pytest.raises(api.TFHEError):
            ctx2.load_keys(tmp_path / "missing.tfhegb")
        # the refused loads left the loaded keys in place
        out = torch.zeros((count, 512), dtype=torch.int32, device="cuda")
        ctx2.bootstrap_gates(api.to_device(ops), dev[0], dev[1], out)
        assert torch.equal(out, outs[0])
    finally:
        ctx2.close()
    ctx3 = api.Context(synth.TFHEParams(n=16))
    try:
        with pytest.raises(api.TFHEError) as err:
            ctx3.load_keys(path)
        assert err.value.code == -1
    finally:
        ctx3.close()


def test_trivial_keys_exact_rotation_large_batch(orc):
    """Zero-mask, zero-noise bootstrapping key: after blind rotation the
    extracted sample is exactly (0, coefficient 0 of X^m v) for every gate of
    a batch larger than the persistent grid."""
    import torch
    from paper_2005_01945_gb300 import api
    p = synth.TFHEParams()
    kd = synth.key_draws(p, 99, noiseless=True, zero_bk_mask=True)
    d = api.to_device
    bk, ksk = api.keygen(p, d(kd.s), d(kd.S), d(kd.bk_mask), d(kd.bk_noise), d(kd.ksk_mask),
                         d(kd.ksk_noise))
    ctx = api.Context(p)
    ctx.set_keys(bk, ksk)
    count = 3001
    rng = np.random.default_rng(5)
    ct = rng.integers(0, M32, size=(count, 512), dtype=np.uint64).astype(np.uint32)
    ct[:, p.n + 1:] = 0
    big = torch.zeros((count, 1056), dtype=torch.int32, device="cuda")
    ctx.blind_rotate_extract(None, d(ct), None, big)
    got = _u32(big)
    abar = orc.modswitch(ct[:, :p.n + 1].reshape(-1), p.N).reshape(count, p.n + 1).astype(np.int64)
    m = ((abar[:, :p.n] * kd.s).sum(axis=1) - abar[:, p.n]) % (2 * p.N)
    coef0 = np.array([trivial_rotation(MU, p.N, int(mm))[0] for mm in m], dtype=np.uint32)
    assert not got[:, :p.N].any()
    assert np.array_equal(got[:, p.N], coef0)
    ctx.close()


def test_many_gates_decrypt_and_sampled_parity(gpu, orc):
    """A batch of 2000 gates (several persistent-grid rounds): every output
    decrypts to the gate's truth value; 12 sampled outputs are bit-exact."""
    torch, api, p, P, kd = gpu["torch"], gpu["api"], gpu["p"], gpu["P"], gpu["kd"]
    count = 2000
    bits, cts, dev = _fresh(gpu, orc, count, 30, "many")
    ops = synth._gen(30, "ops").integers(0, 6, size=count).astype(np.uint8)
    out = torch.empty((count, 512), dtype=torch.int32, device="cuda")
    gpu["ctx"].bootstrap_gates(api.to_device(ops), dev[0], dev[1], out)
    got = _u32(out)
    a, b = bits[0].astype(int), bits[1].astype(int)
    truth = np.select([ops == 0, ops == 1, ops == 2, ops == 3, ops == 4, ops == 5],
                      [1 - (a & b), a & b, a | b, a ^ b, 1 - (a | b), 1 - (a ^ b)])
    dec = orc.decrypt_bits(P, kd.s, got[:, :p.n + 1])
    assert np.array_equal(dec, truth.astype(np.uint8))
    sample = synth._gen(31, "sample").choice(count, 12, replace=False)
    want = orc.gates(P, gpu["obk"], gpu["oksk"], ops[sample], cts[0][sample], cts[1][sample])
    assert np.array_equal(got[sample, :p.n + 1], want)


@pytest.mark.parametrize("group", [1, 2, 4, 5, 8, 16, 32, 33, 40, 48])
def test_each_lockstep_group_bit_exact(gpu, orc, group):
    """Blind rotation with 1, 2 or 4 bootstraps per CTA (13 gates leave empty
    slots in the last group, and skipped CMux steps in some slots), one per
    4-warp CTA compiled for 5 CTAs per SM (shape 5), with one
    bootstrap spread over 8 warps (shape 8), with one bootstrap on a
    cluster of two CTAs exchanging residues (shape 16), and with two per
    CTA reading the key from bulk-copied shared-memory stages (shape 32) or,
    at the same occupancy, through L1 (shape 33), one bootstrap on 8 warps
    with the key staged (shape 40), and the two-CTA cluster with each
    CTA's half of the key staged (shape 48)."""
    torch, api, p, P = gpu["torch"], gpu["api"], gpu["p"], gpu["P"]
    count = 13
    bits, cts, dev = _fresh(gpu, orc, count, 40 + group, f"grp{group}", zero_some=True)
    ops = ((np.arange(count) * 5) % 6).astype(np.uint8)
    out = torch.zeros((count, 512), dtype=torch.int32, device="cuda")
    gpu["ctx"].set_option(api.OPT_BR_GROUP, group)
    try:
        gpu["ctx"].bootstrap_gates(api.to_device(ops), dev[0], dev[1], out)
    finally:
        gpu["ctx"].set_option(api.OPT_BR_GROUP, 0)
    want = orc.gates(P, gpu["obk"], gpu["oksk"], ops, cts[0], cts[1])
    assert np.array_equal(_u32(out)[:, :p.n + 1], want)


@pytest.mark.parametrize("group", [32, 40, 8])
def test_staged_key_across_groups(gpu, orc, group):
    """700 gates on the key-staging shapes (two 4-warp bootstraps per CTA,
    or one on 8 warps) and on the unstaged 8-warp shape: every CTA runs
    several groups, so the staged buffers, their mbarriers and the 8-warp
    shapes' named barriers and exchange rows carry over from group to
    group.  Every output equals the default shape's, and sampled ones the
    oracle's."""
    torch, api, p, P = gpu["torch"], gpu["api"], gpu["p"], gpu["P"]
    count = 700
    bits, cts, dev = _fresh(gpu, orc, count, 91, f"stg{group}")
    ops = ((np.arange(count) * 3) % 6).astype(np.uint8)
    ref = torch.zeros((count, 512), dtype=torch.int32, device="cuda")
    got = torch.zeros((count, 512), dtype=torch.int32, device="cuda")
    gpu["ctx"].bootstrap_gates(api.to_device(ops), dev[0], dev[1], ref)
    gpu["ctx"].set_option(api.OPT_BR_GROUP, group)
    try:
        gpu["ctx"].bootstrap_gates(api.to_device(ops), dev[0], dev[1], got)
    finally:
        gpu["ctx"].set_option(api.OPT_BR_GROUP, 0)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    assert gpu["ctx"].status() == 0
    idx = np.array([0, 151, 152, 303, 304, 305, 699])
    want = orc.gates(P, gpu["obk"], gpu["oksk"], ops[idx], cts[0][idx], cts[1][idx])
    assert np.array_equal(_u32(got)[idx, :p.n + 1], want)


def test_autotune_keeps_results(gpu, orc):
    """Autotuning changes launch shapes only: outputs before and after are
    identical (and equal to the oracle)."""
    torch, api, p, P = gpu["torch"], gpu["api"], gpu["p"], gpu["P"]
    count = 21
    bits, cts, dev = _fresh(gpu, orc, count, 77, "tune")
    ops = ((np.arange(count) * 7) % 6).astype(np.uint8)
    before = torch.zeros((count, 512), dtype=torch.int32, device="cuda")
    after = torch.zeros_like(before)
    gpu["ctx"].bootstrap_gates(api.to_device(ops), dev[0], dev[1], before)
    choices = gpu["ctx"].autotune()
    assert set(choices["br_group"].values()) <= {1, 2, 4, 8, 16, 32, 40, 48}
    assert set(choices["ks_chunks"].values()) <= {1, 2, 4, 8, 16, 32, api.KS_TILED}
    gpu["ctx"].bootstrap_gates(api.to_device(ops), dev[0], dev[1], after)
    assert torch.equal(before, after)
    want = orc.gates(P, gpu["obk"], gpu["oksk"], ops, cts[0], cts[1])
    assert np.array_equal(_u32(after)[:, :p.n + 1], want)
