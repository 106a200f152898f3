"""The allocation-free gate bootstrap (tfhe_bootstrap_gates_noalloc) gives
exactly the same ciphertexts as tfhe_bootstrap_gates.

It exists for callers that cannot let the library allocate device memory
during a call (pre-reserved memory budgets, allocation-free serving loops).
Its scratch is a fixed array shared by all calls on the device, so the
test runs it twice in a row on different inputs (the second call must not
depend on what the first left behind) and checks an oversize batch is
refused.  The file sorts last so a stop-at-first-failure run has already
run every other test."""
import numpy as np
import pytest

from paper_2005_01945_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2005_01945_gb300 import api, build
    build.build()
    p = synth.TFHEParams()
    kd = synth.key_draws(p, 4242)
    d = api.to_device
    bk, ksk = api.keygen(p, d(kd.s), d(kd.S), d(kd.bk_mask), d(kd.bk_noise), d(kd.ksk_mask),
                         d(kd.ksk_noise))
    ctx = api.Context(p)
    ctx.set_keys(bk, ksk)
    yield torch, api, p, kd, ctx
    ctx.close()


def _batch(api, p, kd, count, seed):
    d = api.to_device
    bits = synth.random_bits((2, count), seed, "na")
    cd = synth.ct_draws(p, (2, count), seed, "na")
    s_dev = d(kd.s)
    a = api.encrypt_bits(p, s_dev, d(cd.mask[0]), d(cd.noise[0]), d(bits[0]))
    b = api.encrypt_bits(p, s_dev, d(cd.mask[1]), d(cd.noise[1]), d(bits[1]))
    ops = d(synth._gen(seed, "na_ops").integers(0, 6, size=count).astype(np.uint8))
    return ops, a, b


def test_noalloc_matches_regular_entry_point_twice(env):
    torch, api, p, kd, ctx = env
    for call, (count, seed) in enumerate([(300, 1), (api.NOALLOC_MAX_GATES, 2)]):
        ops, a, b = _batch(api, p, kd, count, seed)
        ref = torch.empty((count, api.LWE_STRIDE), dtype=torch.int32, device="cuda")
        got = torch.full((count, api.LWE_STRIDE), -1, dtype=torch.int32, device="cuda")
        ctx.bootstrap_gates(ops, a, b, ref)
        ctx.bootstrap_gates_noalloc(ops, a, b, got)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), f"call {call}: outputs differ"
        assert ctx.status() == 0


def test_noalloc_rejects_oversize_batch(env):
    torch, api, p, kd, ctx = env
    count = api.NOALLOC_MAX_GATES + 1
    ops, a, b = _batch(api, p, kd, count, 3)
    out = torch.empty((count, api.LWE_STRIDE), dtype=torch.int32, device="cuda")
    with pytest.raises(api.TFHEError) as ei:
        ctx.bootstrap_gates_noalloc(ops, a, b, out)
    assert ei.value.code == -1 and "TFHE_NOALLOC_MAX_GATES" in str(ei.value)
