"""Serving (continuous batching) through the C ABI: requests of mixed kinds
and widths submitted while others run; every result is bit-identical to the
same request run alone and to the oracle (n = 16 ring-size-1024 parameters
so the oracle is quick, and a mix of every served kind at full parameters,
n = 500), and a pool budget smaller than the mix forces requests to wait
for rows without changing any result.  Cancelled requests (queued or
running) never write their outputs and give their rows back to the
pool."""
import concurrent.futures as cf
import threading
import time

import numpy as np
import pytest

from conftest import oparams
from paper_2005_01945_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(orc):
    import torch
    from paper_2005_01945_gb300 import api, build
    build.build()
    p = synth.TFHEParams(n=16)
    P = oparams(p)
    kd = synth.key_draws(p, 71)
    d = api.to_device
    bk, ksk = api.keygen(p, d(kd.s), d(kd.S), d(kd.bk_mask), d(kd.bk_noise), d(kd.ksk_mask),
                         d(kd.ksk_noise))
    obk = orc.keygen_bk(P, kd.s, kd.S, kd.bk_mask, kd.bk_noise)
    oksk = orc.keygen_ksk(P, kd.s, kd.S, kd.ksk_mask, kd.ksk_noise)
    yield dict(torch=torch, api=api, p=p, P=P, kd=kd, bk=bk, ksk=ksk, obk=obk, oksk=oksk)


def _requests(env, seed):
    """A mix: (kind, width, rows, cols, dev in0, dev in1, host in0, host in1, out shape)."""
    api, p, P, kd, orc = env["api"], env["p"], env["P"], env["kd"], __import__("oracle")
    d = api.to_device
    s_dev = d(kd.s)
    rng = np.random.default_rng(seed)
    kinds = [(api.GATE, api.XOR, 0, 0), (api.GATE, api.NAND, 0, 0), (api.ADD, 4, 0, 0),
             (api.ADD, 8, 0, 0), (api.ADD, 16, 0, 0), (api.MUL, 4, 0, 0), (api.MUL, 6, 0, 0),
             (api.MATVEC, 3, 2, 3)]
    reqs = []
    for k in range(24):
        kind, w, r, c = kinds[rng.integers(len(kinds))]
        if kind == api.MATVEC:
            shp0, shp1, outshape = (r, c, w), (c, w), (r, w)
        elif kind == api.GATE:
            shp0, shp1, outshape = (1,), (1,), (1,)
        else:
            shp0, shp1, outshape = (w,), (w,), (w,)
        bits = [synth.random_bits(shp, seed * 100 + k, f"in{j}") for j, shp in enumerate((shp0, shp1))]
        cds = [synth.ct_draws(p, b.shape, seed * 100 + k, f"in{j}") for j, b in enumerate(bits)]
        dev = [api.encrypt_bits(p, s_dev, d(cd.mask), d(cd.noise), d(b)) for cd, b in zip(cds, bits)]
        host = [orc.encrypt_bits(P, kd.s, cd.mask, cd.noise, b) for cd, b in zip(cds, bits)]
        reqs.append((kind, w, r, c, dev[0], dev[1], host[0], host[1], outshape))
    return reqs


def _oracle(env, req):
    orc, api = __import__("oracle"), env["api"]
    kind, w, r, c, _, _, h0, h1, _ = req
    P, bk, ksk = env["P"], env["obk"], env["oksk"]
    if kind == api.GATE:
        return orc.gates(P, bk, ksk, np.array([w], np.uint8), h0, h1)
    if kind == api.ADD:
        return orc.add(P, bk, ksk, w, h0[None], h1[None])[0][0]
    if kind == api.MUL:
        return orc.mul(P, bk, ksk, w, h0[None], h1[None])[0][0]
    return orc.matvec(P, bk, ksk, w, h0, h1)[0]


def _serve(env, reqs, budget, max_batch=0, spacing_s=0.0, threads=1, free_hbm=0):
    torch, api, p = env["torch"], env["api"], env["p"]
    ctx = api.Context(p)
    ctx.set_keys(env["bk"], env["ksk"])
    if free_hbm:
        ctx.set_option(api.OPT_TEST_FREE_HBM, free_hbm)
    outs = [torch.zeros(req[8] + (api.LWE_STRIDE,), dtype=torch.int32, device="cuda") for req in reqs]
    torch.cuda.synchronize()
    ctx.serve_start(budget, max_batch)
    ids = [None] * len(reqs)

    def submit(part):
        for k in part:
            kind, w, r, c, d0, d1 = reqs[k][:6]
            ids[k] = ctx.serve_submit(kind, w, d0, d1, outs[k], r, c)
            if spacing_s:
                time.sleep(spacing_s)

    parts = [list(range(t, len(reqs), threads)) for t in range(threads)]
    ths = [threading.Thread(target=submit, args=(pt,)) for pt in parts]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    lat = [ctx.serve_wait(i, 120000) for i in ids]
    stats = ctx.serve_stats()
    ctx.serve_stop()
    torch.cuda.synchronize()
    res = [o.cpu().numpy().view(np.uint32)[..., :p.n + 1] for o in outs]
    ctx.close()
    return res, lat, stats


def test_mix_equals_alone_and_oracle(env):
    reqs = _requests(env, 5)
    mixed, lat, stats = _serve(env, reqs, budget=256 << 20, spacing_s=0.002, threads=3)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["iterations"] < sum(1 for _ in reqs) * 40   # levels were shared
    assert all(x > 0 for x in lat)
    for k, req in enumerate(reqs):
        alone, _, _ = _serve(env, [req], budget=64 << 20)
        assert np.array_equal(mixed[k], alone[0]), k
        want = _oracle(env, req)
        assert np.array_equal(mixed[k].reshape(want.shape), want), k


def test_small_pool_forces_queueing(env):
    """A pool that holds only a few requests at a time: requests wait for
    rows (continuous admission) and every result is unchanged."""
    reqs = _requests(env, 6)
    roomy, _, _ = _serve(env, reqs, budget=256 << 20)
    tight, _, stats = _serve(env, reqs, budget=400 * 2048, max_batch=64)
    assert stats["completed"] == len(reqs)
    for a, b in zip(roomy, tight):
        assert np.array_equal(a, b)


def _mul16_requests(env, seed, count):
    api, p, P, kd, orc = env["api"], env["p"], env["P"], env["kd"], __import__("oracle")
    d = api.to_device
    s_dev = d(kd.s)
    reqs = []
    for k in range(count):
        bits = [synth.random_bits((16,), seed * 100 + k, f"gm{j}") for j in range(2)]
        cds = [synth.ct_draws(p, b.shape, seed * 100 + k, f"gm{j}") for j, b in enumerate(bits)]
        dev = [api.encrypt_bits(p, s_dev, d(cd.mask), d(cd.noise), d(b)) for cd, b in zip(cds, bits)]
        host = [orc.encrypt_bits(P, kd.s, cd.mask, cd.noise, b) for cd, b in zip(cds, bits)]
        reqs.append((api.MUL, 16, 0, 0, dev[0], dev[1], host[0], host[1], (16,)))
    return reqs


def test_pool_grows_from_free_hbm_and_waits_when_short(env):
    """Admission by free device memory.  Twelve 16-bit multiplications (680
    pool rows of 2 KB each) submitted at once outgrow the pool's first 8 MB:
    the pool maps more device memory and admits them while others run.
    With the device's free memory reported as 1 byte (test hook), the pool
    cannot grow, so requests wait for the rows of finished ones; every
    result is the same either way, and equal to the oracle's."""
    reqs = _mul16_requests(env, 7, 12)
    grown, _, st_g = _serve(env, reqs, budget=1 << 30)
    assert st_g["completed"] == len(reqs) and st_g["failed"] == 0
    assert st_g["pool_grows"] >= 1 and st_g["pool_bytes"] > (8 << 20)
    assert st_g["pool_cap_bytes"] >= (1 << 30)
    assert st_g["admitted_busy"] >= 1
    short, _, st_s = _serve(env, reqs, budget=1 << 30, free_hbm=1)
    assert st_s["completed"] == len(reqs) and st_s["failed"] == 0
    assert st_s["pool_grows"] == 0 and st_s["pool_bytes"] < st_g["pool_bytes"]
    for a, b in zip(grown, short):
        assert np.array_equal(a, b)
    for k in (0, 11):
        want = _oracle(env, reqs[k])
        assert np.array_equal(grown[k], want)


def test_wait_timeout_then_result(env):
    """A client wait that runs out is reported, not hung: waiting 1 ms on a
    16-bit multiplication (56 levels, well over 1 ms) raises TFHE_ETIMEOUT;
    the request keeps running and a second wait returns its result, equal
    to the oracle's."""
    torch, api, p, P, kd = env["torch"], env["api"], env["p"], env["P"], env["kd"]
    orc = __import__("oracle")
    d = api.to_device
    s_dev = d(kd.s)
    bits = [synth.random_bits((16,), 91, f"to{j}") for j in range(2)]
    cds = [synth.ct_draws(p, b.shape, 91, f"to{j}") for j, b in enumerate(bits)]
    dev = [api.encrypt_bits(p, s_dev, d(cd.mask), d(cd.noise), d(b)) for cd, b in zip(cds, bits)]
    host = [orc.encrypt_bits(P, kd.s, cd.mask, cd.noise, b) for cd, b in zip(cds, bits)]
    out = torch.zeros((16, 512), dtype=torch.int32, device="cuda")
    ctx = api.Context(p)
    ctx.set_keys(env["bk"], env["ksk"])
    try:
        ctx.serve_start(64 << 20)
        rid = ctx.serve_submit(api.MUL, 16, dev[0], dev[1], out)
        with pytest.raises(api.TFHEError) as err:
            ctx.serve_wait(rid, 1)
        assert err.value.code == -4          # TFHE_ETIMEOUT
        ctx.serve_wait(rid, 120000)
        ctx.serve_stop()
        want, _ = orc.mul(P, env["obk"], env["oksk"], 16, host[0][None], host[1][None])
        got = out.cpu().numpy().view(np.uint32)[:, :p.n + 1]
        assert np.array_equal(got, want[0])
    finally:
        ctx.close()


def _one_request(env, kind, w, seed):
    """One request of `kind` (opcode `w` for a gate, else the bit width) on
    uniform random operands, encrypted on the device and on the host."""
    api, p, P, kd, orc = env["api"], env["p"], env["P"], env["kd"], __import__("oracle")
    d = api.to_device
    s_dev = d(kd.s)
    nb = 1 if kind == api.GATE else w
    bits = [synth.random_bits((nb,), seed, f"cx{j}") for j in range(2)]
    cds = [synth.ct_draws(p, b.shape, seed, f"cx{j}") for j, b in enumerate(bits)]
    dev = [api.encrypt_bits(p, s_dev, d(cd.mask), d(cd.noise), d(b)) for cd, b in zip(cds, bits)]
    host = [orc.encrypt_bits(P, kd.s, cd.mask, cd.noise, b) for cd, b in zip(cds, bits)]
    return (kind, w, 0, 0, dev[0], dev[1], host[0], host[1], (nb,))


def test_cancel_queued_and_running(env):
    """Cancelling requests.  A pool capped at 3,000 rows holds one 32-bit
    multiplication (2,888 rows) and nothing beside it, so a 16-bit
    multiplication and a gate submitted after it queue, in that order.  The
    gate is cancelled while queued and the 32-bit multiplication while it
    runs (it has 120 levels; the cancel comes within a few of them).
    Neither output buffer is ever written, both report TFHE_ECANCELED, and
    the running request's rows go back to the pool: the 16-bit
    multiplication is admitted into them and completes, equal to the
    oracle.  A finished, an already cancelled or an unknown request cannot
    be cancelled."""
    torch, api, p = env["torch"], env["api"], env["p"]
    reqs = [_one_request(env, api.MUL, 32, 501), _one_request(env, api.MUL, 16, 502),
            _one_request(env, api.GATE, api.AND, 503)]
    sentinel = -12345
    outs = [torch.full(req[8] + (api.LWE_STRIDE,), sentinel, dtype=torch.int32, device="cuda")
            for req in reqs]
    torch.cuda.synchronize()
    ctx = api.Context(p)
    ctx.set_keys(env["bk"], env["ksk"])
    try:
        ctx.serve_start(3000 * api.LWE_STRIDE * 4)
        ids = [ctx.serve_submit(r[0], r[1], r[4], r[5], o, r[2], r[3])
               for r, o in zip(reqs, outs)]
        ctx.serve_cancel(ids[2])                  # queued behind the 16-bit multiplication
        deadline = time.time() + 10.0
        while ctx.serve_stats()["in_flight"] == 0 and time.time() < deadline:
            time.sleep(1e-4)
        assert ctx.serve_stats()["in_flight"] == 1
        ctx.serve_cancel(ids[0])                  # admitted and running
        for k in (0, 2):
            with pytest.raises(api.TFHEError) as err:
                ctx.serve_wait(ids[k], 10000)
            assert err.value.code == -7           # TFHE_ECANCELED
            assert ctx.serve_poll(ids[k])[0] == -7
        ctx.serve_wait(ids[1], 120000)
        for rid in (ids[0], ids[1], 10 ** 9):     # cancelled, completed, unknown
            with pytest.raises(api.TFHEError) as err:
                ctx.serve_cancel(rid)
            assert err.value.code == -1           # TFHE_EINVAL
        st = ctx.serve_stats()
        ctx.serve_stop()
        torch.cuda.synchronize()
        assert st["submitted"] == 3 and st["completed"] == 1 and st["cancelled"] == 2
        assert st["failed"] == 0 and st["in_flight"] == 0 and st["queued"] == 0
        for k in (0, 2):
            assert bool((outs[k] == sentinel).all()), k
        got = outs[1].cpu().numpy().view(np.uint32)[..., :p.n + 1]
        assert np.array_equal(got, _oracle(env, reqs[1]))
    finally:
        ctx.close()


@pytest.fixture(scope="module")
def full_env(orc):
    """Full parameters (n = 500), keys from the master seed."""
    import torch
    from paper_2005_01945_gb300 import api, build
    build.build()
    p = synth.TFHEParams()
    P = oparams(p)
    kd = synth.key_draws(p, synth.MASTER_SEED)
    d = api.to_device
    bk, ksk = api.keygen(p, d(kd.s), d(kd.S), d(kd.bk_mask), d(kd.bk_noise), d(kd.ksk_mask),
                         d(kd.ksk_noise))
    obk = orc.keygen_bk(P, kd.s, kd.S, kd.bk_mask, kd.bk_noise)
    oksk = orc.keygen_ksk(P, kd.s, kd.S, kd.ksk_mask, kd.ksk_noise)
    yield dict(torch=torch, api=api, p=p, P=P, kd=kd, bk=bk, ksk=ksk, obk=obk, oksk=oksk)


def _full_requests(env, seed):
    """One request of every kind the served workload draws from (single gate,
    16- and 32-bit addition, 16- and 32-bit multiplication), plus a second
    gate and 16-bit addition, on uniform random operands."""
    api, p, P, kd, orc = env["api"], env["p"], env["P"], env["kd"], __import__("oracle")
    d = api.to_device
    s_dev = d(kd.s)
    kinds = [(api.GATE, api.XOR), (api.ADD, 16), (api.MUL, 32), (api.ADD, 32), (api.MUL, 16),
             (api.GATE, api.AND), (api.ADD, 16)]
    reqs = []
    for k, (kind, w) in enumerate(kinds):
        nb = 1 if kind == api.GATE else w
        bits = [synth.random_bits((nb,), seed * 100 + k, f"fin{j}") for j in range(2)]
        cds = [synth.ct_draws(p, b.shape, seed * 100 + k, f"fin{j}") for j, b in enumerate(bits)]
        dev = [api.encrypt_bits(p, s_dev, d(cd.mask), d(cd.noise), d(b)) for cd, b in zip(cds, bits)]
        host = [orc.encrypt_bits(P, kd.s, cd.mask, cd.noise, b) for cd, b in zip(cds, bits)]
        reqs.append((kind, w, 0, 0, dev[0], dev[1], host[0], host[1], (nb,)))
    return reqs


def test_full_parameters_mix_equals_alone_and_oracle(full_env):
    """Served mix at full parameters (n = 500): requests of every kind are
    submitted from three threads while others run, so they share levels on
    the device.  Each result equals the same request served alone and the
    oracle's ciphertexts word for word (recomputed gate by gate, the 32-bit
    multiplication 2,824 bootstraps and 120 levels deep), and the 32-bit
    multiplication decrypts to the product."""
    env = full_env
    api, orc = env["api"], __import__("oracle")
    reqs = _full_requests(env, 17)
    mixed, lat, stats = _serve(env, reqs, budget=512 << 20, spacing_s=0.003, threads=3)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert all(x > 0 for x in lat)
    alone = [_serve(env, [req], budget=128 << 20)[0][0] for req in reqs]
    for k in range(len(reqs)):
        assert np.array_equal(mixed[k], alone[k]), k
    checked = list(range(len(reqs)))
    with cf.ThreadPoolExecutor(len(checked)) as ex:
        wants = list(ex.map(lambda k: _oracle(env, reqs[k]), checked))
    for k, want in zip(checked, wants):
        assert np.array_equal(mixed[k].reshape(want.shape), want), k
    k32 = next(k for k, r in enumerate(reqs) if r[0] == api.MUL and r[1] == 32)
    bits = orc.decrypt_bits(env["P"], env["kd"].s, mixed[k32])
    a = synth.from_bits(orc.decrypt_bits(env["P"], env["kd"].s, reqs[k32][6])[None])[0]
    b = synth.from_bits(orc.decrypt_bits(env["P"], env["kd"].s, reqs[k32][7])[None])[0]
    assert synth.from_bits(bits[None])[0] == (int(a) * int(b)) % (1 << 32)
