"""The allocation-free gate bootstrap (tfhe_bootstrap_gates_noalloc) gives
exactly the same ciphertexts as tfhe_bootstrap_gates.

It exists for callers that cannot let the library allocate device memory
during a call (pre-reserved memory budgets, allocation-free serving loops).
Its scratch is a fixed array shared by all calls on the device, so the
test runs it several times in a row on different inputs, the larger call
first (a later call must not depend on what an earlier one left behind),
once on a side stream and once with another key-switch kernel chosen, and
checks that an oversize batch is refused.  The file sorts last so a stop-at-first-failure run has already
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


def _compare(torch, api, ctx, ops, a, b, stream=None):
    count = ops.numel()
    ref = torch.empty((count, api.LWE_STRIDE), dtype=torch.int32, device="cuda")
    got = torch.full((count, api.LWE_STRIDE), -1, dtype=torch.int32, device="cuda")
    ctx.bootstrap_gates(ops, a, b, ref)
    torch.cuda.synchronize()
    before = ctx.launches()
    if stream is None:
        ctx.bootstrap_gates_noalloc(ops, a, b, got)
    else:
        with torch.cuda.stream(stream):
            ctx.bootstrap_gates_noalloc(ops, a, b, got, stream=stream)
    torch.cuda.synchronize()
    return torch.equal(got, ref), ctx.launches() - before


def test_noalloc_matches_regular_entry_point_in_a_row(env):
    """A full-size call, then smaller ones: the smaller calls read rows of
    the shared array that the larger call left behind, so they show that
    nothing in it needs clearing.  The last call runs on a side stream."""
    torch, api, p, kd, ctx = env
    side = torch.cuda.Stream()
    plan = [(api.NOALLOC_MAX_GATES, 2, None), (300, 1, None), (37, 5, side)]
    for call, (count, seed, stream) in enumerate(plan):
        ops, a, b = _batch(api, p, kd, count, seed)
        same, _ = _compare(torch, api, ctx, ops, a, b, stream)
        assert same, f"call {call} ({count} gates): outputs differ"
        assert ctx.status() == 0


def test_noalloc_follows_the_key_switch_choice(env):
    """With the direct key-switch kernel forced (TFHE_OPT_KS_KERNEL = 1: one
    launch, where the tiled kernel takes two at this width), the
    allocation-free call launches what tfhe_bootstrap_gates launches and
    gives the same ciphertexts."""
    torch, api, p, kd, ctx = env
    ops, a, b = _batch(api, p, kd, 200, 7)
    counts = {}
    for choice in (1, api.KS_TILED):
        ctx.set_option(api.OPT_KS_KERNEL, choice)
        try:
            torch.cuda.synchronize()
            before = ctx.launches()
            ref = torch.empty((200, api.LWE_STRIDE), dtype=torch.int32, device="cuda")
            ctx.bootstrap_gates(ops, a, b, ref)
            regular = ctx.launches() - before
            same, noalloc = _compare(torch, api, ctx, ops, a, b)
        finally:
            ctx.set_option(api.OPT_KS_KERNEL, 0)
        assert same, f"key-switch choice {choice}: outputs differ"
        assert noalloc == regular, f"key-switch choice {choice}: {noalloc} vs {regular} launches"
        counts[choice] = noalloc
    assert counts[1] < counts[api.KS_TILED]
    assert ctx.status() == 0


def test_noalloc_rejects_oversize_batch(env):
    torch, api, p, kd, ctx = env
    count = api.NOALLOC_MAX_GATES + 1
    ops, a, b = _batch(api, p, kd, count, 3)
    out = torch.empty((count, api.LWE_STRIDE), dtype=torch.int32, device="cuda")
    with pytest.raises(api.TFHEError) as ei:
        ctx.bootstrap_gates_noalloc(ops, a, b, out)
    assert ei.value.code == -1 and "TFHE_NOALLOC_MAX_GATES" in str(ei.value)
