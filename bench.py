#!/usr/bin/env python3
"""Benchmark: bootstrapped gates per second on one GB300.

Workload (one step): a batch of 256 homomorphic 32-bit ripple-carry
additions of uniform random operands encrypted bitwise with TFHE (LWE
n=500, TLWE N=1024, Bg=2^10, l=2, key switch t=8, base 4): 154 bootstrapped
gates each, 39,424 per step, scheduled as 62 levels of batched bootstraps
replayed as one CUDA graph.  Also reported: the other full-size workloads
(64 + 64 multiplications of 16 and 32 bits in one schedule; the 16x16
matrix-vector product) with their own blind-rotation roofline,
single-request 32-bit multiplication latency (p50/p99 over 50 runs),
level-batched versus one launch pair per gate, and the CPU oracle's gate
rate on the host cores (all cores and one thread).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs the same workload on its own GPU
(replicas, no collective on the data path); value counts all ranks' gates
over the slowest rank's time.  ``--impl reference`` times the CPU oracle
(rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "bootstrapped gates/sec on 1 GB300; 32-bit enc. mul p50/p99 latency, batched vs per-gate"
WORKLOAD = ("256 homomorphic 32-bit ripple-carry additions per step (39,424 bootstrapped gates, "
            "62 levels); TFHE LWE n=500, TLWE N=1024 k=1, Bg=2^10 l=2, key switch t=8 base 4, "
            "Torus32; keys, noise and operands from one seed")
BATCH, WIDTH = 256, 32
GATES_PER_ADD = 5 * WIDTH - 6

# Algorithmic 32-bit integer operations of one CMux step of the NTT-based
# external product: 12 transforms of
# 5120 radix-2 butterflies at 7 ops, 12 x 1024 twiddle products at 3 ops,
# 2 x 2 x 1024 pointwise 4-term products at 12 ops, 4 x 1024 digit
# extractions at 8 ops, 2 x 1024 CRT lifts + accumulates at 12 ops.
OPS_PER_CMUX = 12 * 5120 * 7 + 12 * 1024 * 3 + 4 * 1024 * 12 + 4 * 1024 * 8 + 2 * 1024 * 12
INT32_LANES_PER_SM = 128
# Key-switching key as the algorithm reads it: N x t x (base - 1) LWE rows of
# n + 1 words (the padding to 512 words is layout, not algorithm).
KSK_BYTES = 1024 * 8 * 3 * 501 * 4


def max_over_ranks(value, dist, device=None):
    """Largest value over all ranks (the slowest rank's time)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_step, steps, world, max_ms):
    """Units all ranks processed divided by the slowest rank's time (s)."""
    return units_per_step * steps * world / (max_ms / 1e3)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--latency-samples", type=int, default=50,
                    help="level-batched 32-bit multiplications timed per multiplier")
    ap.add_argument("--per-gate-samples", type=int, default=3,
                    help="one-launch-pair-per-gate runs of the sequential multiplier")
    ap.add_argument("--per-gate-samples-shallow", type=int, default=10,
                    help="one-launch-pair-per-gate runs of the Dadda multiplier")
    ap.add_argument("--product-choice", type=int, default=2432,
                    help="bootstraps of the tensor-pipe vs NTT CMux comparison in the bench line "
                         "(a multiple of 128; 0: skip)")
    ap.add_argument("--config-steps", type=int, default=3,
                    help="timed steps of configs 2 and 3 (after one warm-up step)")
    ap.add_argument("--cpu-gates-single", type=int, default=8,
                    help="oracle gates timed on one host thread")
    ap.add_argument("--no-latency", action="store_true")
    ap.add_argument("--cpu-gates", type=int, default=128)
    ap.add_argument("--br-only", type=int, default=0, help="profile mode: blind rotation alone")
    ap.add_argument("--br-group", type=int, default=0, help="blind-rotation CTA shape: 1, 2, 4 bootstraps per CTA, 8 = one "
                         "bootstrap on 8 warps, 16 = one bootstrap on two CTAs (0: automatic)")
    ap.add_argument("--ks-only", type=int, default=0,
                    help="profile mode: key switch alone on this many uniform LWE_N samples")
    ap.add_argument("--tc-products", type=int, default=0,
                    help="measure the tensor-pipe CMux products (count bootstraps, a multiple "
                         "of 128) against the NTT blind rotation")
    ap.add_argument("--ks-kernel", type=int, default=0,
                    help="key-switch kernel: 64 tiled, 1..32 direct with that j-split (0: default)")
    ap.add_argument("--serve", action="store_true",
                    help="serving workload: Poisson requests at 3 rates (config 4)")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-sample", type=int, default=400,
                    help="requests per arrival rate of the bounded config-4 serving measurement "
                         "in the bench line (0: skip)")
    ap.add_argument("--serve-circuits", default="paper", choices=["paper", "shallow"],
                    help="serving circuits: the paper's ripple-carry adders and shift-and-add "
                         "multipliers, or parallel-prefix adders and Dadda-tree multipliers "
                         "(same results, fewer levels)")
    ap.add_argument("--variants", action="store_true",
                    help="adder / multiplier variants and the compound-gate ablation")
    ap.add_argument("--configs", action="store_true",
                    help="time configs 0 (8 gates), 2 (mul16/mul32 x64) and 3 (matvec 16x16)")
    ap.add_argument("--config-set", default="0,2,3",
                    help="with --configs: which of the configs 0, 2 and 3 to run (comma list)")
    ap.add_argument("--tune-cache", default=None,
                    help="autotuner cache file (read if present, appended after tuning)")
    return ap.parse_args()


KERNEL_SOURCES = ("paper_2005_01945_gb300/csrc/bootstrap.cu",
                  "paper_2005_01945_gb300/csrc/common.cuh")
TRAFFIC_PROFILE = "profiles/k_blind_rotate_traffic_add32x256.md"


def kernel_source_sha1():
    import hashlib
    h = hashlib.sha1()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def br_traffic_per_launch():
    """DRAM bytes per blind-rotation launch from the committed ncu capture,
    or None when the kernel sources changed since it was taken."""
    try:
        fields = {}
        for line in open(os.path.join(ROOT, TRAFFIC_PROFILE)):
            line = line.strip().lstrip("-* ")
            if ":" in line and line.startswith(("bytes_per_launch", "kernel_source_sha1")):
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
        if fields.get("kernel_source_sha1") != kernel_source_sha1():
            return None
        return float(fields["bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        exe = shutil.which("nvidia-smi")
        if not exe:
            return
        self.f = open(self.path, "w")
        self.proc = subprocess.Popen([exe, f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                      "-lms", "200", "-i", str(self.index)], stdout=self.f,
                                     stderr=subprocess.DEVNULL)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                mx.append(float(f[2].split()[0]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


class OracleSample:
    """CPU oracle (plain C, OpenMP over gates) on a bounded sample of the
    workload: the first-level gates (XOR / AND of fresh input bits) of the
    first additions of the batch, each a full bootstrap + key switch."""

    def __init__(self, ngates, seed):
        import oracle
        from paper_2005_01945_gb300 import synth
        self.oracle = oracle
        p = synth.TFHEParams()
        self.P = P = oracle.Params(p.n, p.N, p.l, p.bg_bit, p.ks_t, p.ks_basebit)
        kd = synth.key_draws(p, seed)
        self.bk = oracle.keygen_bk(P, kd.s, kd.S, kd.bk_mask, kd.bk_noise)
        self.ksk = oracle.keygen_ksk(P, kd.s, kd.S, kd.ksk_mask, kd.ksk_noise)
        a, b = synth.int_pairs(BATCH, WIDTH, seed + 1, "add32")
        ba, bb = synth.to_bits(a, WIDTH), synth.to_bits(b, WIDTH)
        cda = synth.ct_draws(p, ba.shape, seed + 1, "add32a")
        cdb = synth.ct_draws(p, bb.shape, seed + 1, "add32b")
        k = np.arange(ngates)
        inst, bit = k // (2 * WIDTH), (k // 2) % WIDTH
        self.op = np.where(k % 2 == 0, 3, 1).astype(np.uint8)
        self.ca = oracle.encrypt_bits(P, kd.s, cda.mask[inst, bit], cda.noise[inst, bit],
                                      ba[inst, bit])
        self.cb = oracle.encrypt_bits(P, kd.s, cdb.mask[inst, bit], cdb.noise[inst, bit],
                                      bb[inst, bit])
        self.ngates = ngates
        self.cores = oracle.max_threads()
        self.desc = (f"{ngates} first-level XOR/AND gates of the 32-bit additions of the batch "
                     f"(full bootstrap + key switch each), OpenMP over gates")

    def rate(self, ngates=None, threads=None):
        k = self.ngates if ngates is None else min(ngates, self.ngates)
        t0 = time.perf_counter()
        self.oracle.gates(self.P, self.bk, self.ksk, self.op[:k], self.ca[:k], self.cb[:k],
                          nthreads=self.cores if threads is None else threads)
        return k / (time.perf_counter() - t0)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2005_01945_gb300 import synth
    sample = OracleSample(max(16, args.cpu_gates // 4), synth.MASTER_SEED)
    for _ in range(args.warmup):
        sample.rate()
    rates = [sample.rate() for _ in range(args.steps)]
    value = statistics.mean(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "gates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sample.ngates / value * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample.desc},
            "cpu_baseline": {"value": value, "unit": "gates/s", "cores": sample.cores,
                             "kind": "oracle", "sample": sample.desc},
            "e2e": {"value": value, "unit": "gates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_br_only(count, group=0):
    """Blind rotation + extraction alone on `count` fresh gates (profiling)."""
    import torch
    from paper_2005_01945_gb300 import api, build, synth
    build.build()
    p = synth.TFHEParams()
    kd = synth.key_draws(p, synth.MASTER_SEED)
    d = api.to_device
    bk, ksk = api.keygen(p, d(kd.s), d(kd.S), d(kd.bk_mask), d(kd.bk_noise), d(kd.ksk_mask),
                         d(kd.ksk_noise))
    ctx = api.Context(p)
    ctx.set_keys(bk, ksk)
    ctx.set_option(api.OPT_BR_GROUP, group)
    bits = synth.random_bits((2, count), 7, "bronly")
    cd = synth.ct_draws(p, (2, count), 7, "bronly")
    s_dev = d(kd.s)
    ca = api.encrypt_bits(p, s_dev, d(cd.mask[0]), d(cd.noise[0]), d(bits[0]))
    cb = api.encrypt_bits(p, s_dev, d(cd.mask[1]), d(cd.noise[1]), d(bits[1]))
    ops = d(np.full(count, 3, np.uint8))
    big = torch.empty((count, api.BIG_STRIDE), dtype=torch.int32, device="cuda")
    out = torch.empty((count, api.LWE_STRIDE), dtype=torch.int32, device="cuda")
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    br, ks = [], []
    for _ in range(3):
        e0.record()
        ctx.blind_rotate_extract(ops, ca, cb, big)
        e1.record()
        ctx.keyswitch(big, out)
        e2.record()
        torch.cuda.synchronize()
        br.append(e0.elapsed_time(e1))
        ks.append(e1.elapsed_time(e2))
    print(json.dumps({"br_only": count, "group": group, "br_ms": br, "ks_ms": ks,
                      "bootstraps_per_s": count / (min(br) / 1e3)}), flush=True)
    ctx.close()


def tc_vs_ntt(ctx, p, kd, count, reps=5, device="cuda"):
    """The exact-product choice, measured: one CMux step's 8 negacyclic
    products on the tensor pipe (tcgen05, limb-split bf16, exact fp32 sums)
    for `count` bootstraps, against the NTT blind rotation of the same count
    (n = 500 CMux steps, each with decomposition, 12 transforms, pointwise
    products, CRT and accumulation), per CMux step and bootstrap."""
    import torch
    from paper_2005_01945_gb300 import api, synth
    g = synth._gen(9, "tc_bench")
    d = lambda a: api.to_device(a, device)  # noqa: E731
    rows = d(g.integers(0, 1 << 32, size=(4, 2, 1024), dtype=np.uint64).astype(np.uint32))
    dig = d(g.integers(-512, 512, size=(count, 4, 1024), dtype=np.int64).astype(np.int32))
    key_ops = torch.empty(api.tc_key_bytes(), dtype=torch.uint8, device=device)
    digit_ops = torch.empty(api.tc_digit_bytes(count), dtype=torch.uint8, device=device)
    out = torch.empty((count, 2, 1024), dtype=torch.int32, device=device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    prep_ms = timed(lambda: ctx.tc_prepare_key(rows, key_ops))
    tc_ms = timed(lambda: ctx.cmux_products_tc(dig, key_ops, digit_ops, out))
    bits = synth.random_bits((2, count), 7, "tcntt")
    cd = synth.ct_draws(p, (2, count), 7, "tcntt")
    s_dev = d(kd.s)
    ca = api.encrypt_bits(p, s_dev, d(cd.mask[0]), d(cd.noise[0]), d(bits[0]))
    cb = api.encrypt_bits(p, s_dev, d(cd.mask[1]), d(cd.noise[1]), d(bits[1]))
    ops = d(np.full(count, 3, np.uint8))
    big = torch.empty((count, api.BIG_STRIDE), dtype=torch.int32, device=device)
    br_ms = timed(lambda: ctx.blind_rotate_extract(ops, ca, cb, big))
    bf16 = float(measured_peaks().get("bf16_tflops", 1900.0))
    flops = 2.0 * 8 * 4096 * 2048 * count          # 8 limb pairs x (M x 4N x 2N)
    tc_best = min(tc_ms)
    ntt_cmux_ns = min(br_ms) * 1e6 / (p.n * count)
    return {"bootstraps": count, "status": ctx.status(),
            "tc_prepare_key_ms": prep_ms, "tc_products_ms": tc_ms,
            "tc_ns_per_cmux_bootstrap": tc_best * 1e6 / count,
            "tc_tflops": flops / (tc_best / 1e3) / 1e12,
            "tc_frac_of_bf16_peak": flops / (tc_best / 1e3) / 1e12 / bf16,
            "tc_ns_per_cmux_bootstrap_at_peak": flops / (bf16 * 1e12) * 1e9 / count,
            "ntt_blind_rotation_ms": br_ms, "ntt_ns_per_cmux_bootstrap": ntt_cmux_ns,
            "tc_over_ntt": (tc_best * 1e6 / count) / ntt_cmux_ns,
            "chosen": "ntt" if tc_best * 1e6 / count > ntt_cmux_ns else "tensor"}


def run_tc_products(count, reps=5):
    """CLI mode of tc_vs_ntt with its own context and keys."""
    from paper_2005_01945_gb300 import api, build, synth
    build.build()
    p = synth.TFHEParams()
    d = api.to_device
    kd = synth.key_draws(p, synth.MASTER_SEED)
    bk, ksk = api.keygen(p, d(kd.s), d(kd.S), d(kd.bk_mask), d(kd.bk_noise), d(kd.ksk_mask),
                         d(kd.ksk_noise))
    ctx = api.Context(p)
    ctx.set_keys(bk, ksk)
    res = tc_vs_ntt(ctx, p, kd, count, reps)
    res["tc_products"] = res.pop("bootstraps")
    print(json.dumps(res), flush=True)
    ctx.close()


def run_ks_only(count, kernel=0):
    """Key switch alone on `count` uniform LWE_N samples (profiling): CUDA
    event times of 5 launches after a warm-up, and the rate of key bytes."""
    import torch
    from paper_2005_01945_gb300 import api, build, synth
    build.build()
    p = synth.TFHEParams()
    kd = synth.key_draws(p, synth.MASTER_SEED)
    d = api.to_device
    bk, ksk = api.keygen(p, d(kd.s), d(kd.S), d(kd.bk_mask), d(kd.bk_noise), d(kd.ksk_mask),
                         d(kd.ksk_noise))
    ctx = api.Context(p)
    ctx.set_keys(bk, ksk)
    ctx.set_option(api.OPT_KS_KERNEL, kernel)
    big = d(synth._gen(11, "ksonly").integers(0, 1 << 32, size=(count, api.BIG_STRIDE),
                                              dtype=np.uint64).astype(np.uint32).view(np.int32))
    out = torch.empty((count, api.LWE_STRIDE), dtype=torch.int32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.keyswitch(big, out)
    ms = []
    for _ in range(5):
        e0.record()
        ctx.keyswitch(big, out)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    alg = KSK_BYTES + count * (p.N + 1 + p.n + 1) * 4
    print(json.dumps({"ks_only": count, "kernel": kernel or "default", "ks_ms": ms,
                      "algorithmic_bytes": alg, "gb_per_s": alg / (min(ms) / 1e3) / 1e9,
                      "status": ctx.status()}), flush=True)
    ctx.close()


def run_variants(args):
    """Circuit variants of the paper (sections V-A, V-B): adders (ripple carry,
    majority carry, number-wise GPU_n), truncated multipliers (sequential,
    tree accumulation) and full products (naive, Karatsuba), as batches and
    as single-request latency; and the
    compound-gate ablation (section V-A-3, Fig. "compoundGateAna"): the XOR
    and AND of two w-bit numbers as two launches or as one."""
    import torch
    from paper_2005_01945_gb300 import api, build, synth
    build.build()
    p = synth.TFHEParams()
    seed = synth.MASTER_SEED + 5
    kd = synth.key_draws(p, seed)
    d = api.to_device
    bk, ksk = api.keygen(p, d(kd.s), d(kd.S), d(kd.bk_mask), d(kd.bk_noise), d(kd.ksk_mask),
                         d(kd.ksk_noise))
    ctx = api.Context(p)
    ctx.set_keys(bk, ksk)
    ctx.autotune(args.tune_cache)
    s_dev = d(kd.s)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def enc(xs, w, tag):
        bits = synth.to_bits(xs, w)
        cd = synth.ct_draws(p, bits.shape, seed, tag)
        return api.encrypt_bits(p, s_dev, d(cd.mask), d(cd.noise), d(bits))

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.median(ms))

    dec = lambda t: synth.from_bits(api.decrypt_bits(p, s_dev, t).cpu().numpy())  # noqa: E731
    res = {"adders_256x32": {}, "multipliers_32": {}, "compound_gate": []}
    a, b = synth.int_pairs(256, 32, seed, "var_add")
    A, B = enc(a, 32, "va"), enc(b, 32, "vb")
    R = torch.empty_like(A)
    for name, kind in (("ripple", api.ADD), ("majority", api.ADD_MAJ), ("numberwise", api.ADD_NW),
                       ("prefix", api.ADD_PREFIX)):
        job = [dict(kind=kind, width=32, batch=256, in0=A, in1=B, out=R)]
        ms = timed(lambda: ctx.run_jobs(job), 3)
        g, depth = api.circuit_info(kind, 32)
        res["adders_256x32"][name] = {"ms": ms, "gates": 256 * g, "depth": depth,
                                      "gates_per_s": 256 * g / (ms / 1e3),
                                      "verified": bool(np.array_equal(dec(R), (a + b) % (1 << 32)))}
        one = [dict(kind=kind, width=32, batch=1, in0=A[:1], in1=B[:1], out=R[:1])]
        res["adders_256x32"][name]["single_ms"] = timed(lambda: ctx.run_jobs(one), 5)
    ma, mb = synth.int_pairs(64, 32, seed, "var_mul")
    MA, MB = enc(ma, 32, "vma"), enc(mb, 32, "vmb")
    MR = torch.empty_like(MA)
    for name, kind in (("sequential", api.MUL), ("tree", api.MUL_TREE),
                       ("tree_maj", api.MUL_TREE_MAJ), ("dadda", api.MUL_DADDA)):
        job = [dict(kind=kind, width=32, batch=64, in0=MA, in1=MB, out=MR)]
        ms = timed(lambda: ctx.run_jobs(job), 2)
        g, depth = api.circuit_info(kind, 32)
        ok = bool(np.array_equal(dec(MR), (ma * mb) % (1 << 32)))
        one = [dict(kind=kind, width=32, batch=1, in0=MA[:1], in1=MB[:1], out=MR[:1])]
        res["multipliers_32"][name] = {"batch64_ms": ms, "gates": 64 * g, "depth": depth,
                                       "gates_per_s": 64 * g / (ms / 1e3),
                                       "single_ms": timed(lambda: ctx.run_jobs(one), 5),
                                       "verified": ok}
    def dec_wide(t):
        bits = api.decrypt_bits(p, s_dev, t).cpu().numpy()
        return [sum(int(v) << i for i, v in enumerate(row)) for row in bits]

    # full products (2w bits): naive with tree accumulation vs Karatsuba
    # (section III-B, Table "multiplicationComparison")
    res["full_products"] = {}
    for w, batch in ((16, 64), (32, 32), (64, 8)):
        fa, fb = synth.int_pairs(batch, w, seed, f"var_full{w}")
        FA, FB = enc(fa, w, f"vfa{w}"), enc(fb, w, f"vfb{w}")
        FR = torch.empty((batch, 2 * w, api.LWE_STRIDE), dtype=torch.int32, device="cuda")
        want = [int(x) * int(y) for x, y in zip(fa, fb)]
        entry = {}
        for name, kind in (("naive", api.MUL_FULL), ("karatsuba", api.MUL_KARATSUBA)):
            job = [dict(kind=kind, width=w, batch=batch, in0=FA, in1=FB, out=FR)]
            ms = timed(lambda: ctx.run_jobs(job), 2)
            ok = dec_wide(FR) == want
            g, depth = api.circuit_info(kind, w)
            one = [dict(kind=kind, width=w, batch=1, in0=FA[:1], in1=FB[:1], out=FR[:1])]
            entry[name] = {f"batch{batch}_ms": ms, "gates": batch * g, "depth": depth,
                           "gates_per_s": batch * g / (ms / 1e3),
                           "single_ms": timed(lambda: ctx.run_jobs(one), 3), "verified": ok}
        res["full_products"][f"{w}x{w}"] = entry
    for w in (1, 2, 4, 8, 16, 32):
        x, y = synth.int_pairs(1, w, seed, f"cg{w}")
        X, Y = enc(x, w, f"cgx{w}")[0], enc(y, w, f"cgy{w}")[0]
        out = torch.empty((2 * w, api.LWE_STRIDE), dtype=torch.int32, device="cuda")
        xor_ops = d(np.full(w, api.XOR, np.uint8))
        and_ops = d(np.full(w, api.AND, np.uint8))
        both = d(np.array([api.XOR] * w + [api.AND] * w, np.uint8))
        XX, YY = torch.cat([X, X]), torch.cat([Y, Y])

        def two():
            ctx.bootstrap_gates(xor_ops, X, Y, out[:w])
            ctx.bootstrap_gates(and_ops, X, Y, out[w:])

        def one():
            ctx.bootstrap_gates(both, XX, YY, out)

        res["compound_gate"].append({"bits": w, "two_launches_ms": timed(two, 5),
                                     "one_launch_ms": timed(one, 5)})
    print(json.dumps({"metric": "circuit variants (sections V-A, V-B)", "results": res}),
          flush=True)
    ctx.close()


def run_configs(args):
    """Throughput of the other workloads (device-resident inputs, CUDA events,
    L2 flushed before every timed run), each verified by decryption."""
    import torch
    from paper_2005_01945_gb300 import api, build, synth
    build.build()
    p = synth.TFHEParams()
    seed = synth.MASTER_SEED
    kd = synth.key_draws(p, seed)
    d = api.to_device
    bk, ksk = api.keygen(p, d(kd.s), d(kd.S), d(kd.bk_mask), d(kd.bk_noise), d(kd.ksk_mask),
                         d(kd.ksk_noise))
    ctx = api.Context(p)
    ctx.set_keys(bk, ksk)
    ctx.autotune(args.tune_cache)
    s_dev = d(kd.s)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def enc(xs, w, tag):
        bits = synth.to_bits(xs, w)
        cd = synth.ct_draws(p, bits.shape, seed, tag)
        return api.encrypt_bits(p, s_dev, d(cd.mask), d(cd.noise), d(bits))

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.median(ms))

    dec = lambda t: synth.from_bits(api.decrypt_bits(p, s_dev, t).cpu().numpy())  # noqa: E731
    chosen = {int(c) for c in args.config_set.split(",") if c.strip()}
    if not chosen or not chosen <= {0, 2, 3}:
        raise SystemExit(f"--config-set: expected a comma list of 0, 2, 3, got {args.config_set!r}")
    out = {}
    if 0 in chosen:
        config0(ctx, d, enc, timed, seed, out)
    if 2 in chosen:
        config2(ctx, api, enc, timed, dec, seed, out)
    if 3 in chosen:
        config3(ctx, api, enc, timed, dec, seed, out)
    print(json.dumps({"metric": "bootstrapped gates/sec per workload", "unit": "gates/s",
                      "results": out}), flush=True)
    ctx.close()


def config0(ctx, d, enc, timed, seed, out):
    """Config 0: 8 gates (NAND, AND, OR, XOR, two each) in one call."""
    import torch
    from paper_2005_01945_gb300 import synth
    ops, ba, bb = synth.gates8_inputs(seed)
    A0, B0 = enc(ba, 1, "c0a")[:, 0], enc(bb, 1, "c0b")[:, 0]
    R0 = torch.empty_like(A0)
    ops_d = d(ops)
    ms = timed(lambda: ctx.bootstrap_gates(ops_d, A0, B0, R0), 10)
    out["config0_8gates"] = {"ms": ms, "gates_per_s": 8 / (ms / 1e3)}


def config2(ctx, api, enc, timed, dec, seed, out):
    """Config 2: 64 mul16 + 64 mul32 in one level schedule."""
    import torch
    from paper_2005_01945_gb300 import synth
    a16, b16 = synth.int_pairs(64, 16, seed + 2, "mul16")
    a32, b32 = synth.int_pairs(64, 32, seed + 2, "mul32")
    A16, B16, A32, B32 = enc(a16, 16, "m16a"), enc(b16, 16, "m16b"), enc(a32, 32, "m32a"), \
        enc(b32, 32, "m32b")
    R16, R32 = torch.empty_like(A16), torch.empty_like(A32)
    jobs = [dict(kind=api.MUL, width=16, batch=64, in0=A16, in1=B16, out=R16),
            dict(kind=api.MUL, width=32, batch=64, in0=A32, in1=B32, out=R32)]
    ms = timed(lambda: ctx.run_jobs(jobs), 3)
    gates = 64 * (api.circuit_info(api.MUL, 16)[0] + api.circuit_info(api.MUL, 32)[0])
    ok = bool(np.array_equal(dec(R16), (a16 * b16) % (1 << 16)) and
              np.array_equal(dec(R32), (a32 * b32) % (1 << 32)))
    out["config2_mul16x64_mul32x64"] = {"ms": ms, "gates": gates,
                                        "gates_per_s": gates / (ms / 1e3), "verified": ok}


def config3(ctx, api, enc, timed, dec, seed, out):
    """Config 3: 16x16 matrix times a length-16 vector, 16-bit words."""
    import torch
    from paper_2005_01945_gb300 import synth
    M = synth.random_uints((16, 16), 16, seed + 3, "M")
    v = synth.random_uints(16, 16, seed + 3, "v")
    MM, vv = enc(M, 16, "M"), enc(v, 16, "v")
    y = torch.empty((16, 16, api.LWE_STRIDE), dtype=torch.int32, device="cuda")
    ms = timed(lambda: ctx.matvec(16, MM, vv, y), 3)
    gates = api.circuit_info(api.MATVEC, 16, 16, 16)[0]
    ok = bool(np.array_equal(dec(y), (M * v[None, :]).sum(axis=1) % (1 << 16)))
    out["config3_matvec16"] = {"ms": ms, "gates": gates, "gates_per_s": gates / (ms / 1e3),
                               "verified": ok}


SERVE_KINDS = [("gate", 0, 1), ("add16", 1, 16), ("add32", 1, 32), ("mul16", 2, 16),
               ("mul32", 2, 32)]
# the same requests with the shallow circuits (ADD_PREFIX = 10, MUL_DADDA = 11)
SERVE_KINDS_SHALLOW = [("gate", 0, 1), ("add16", 10, 16), ("add32", 10, 32), ("mul16", 11, 16),
                       ("mul32", 11, 32)]


def measure_serving(ctx, p, s_dev, d, seed, table, per_rate, burst=200):
    """Config 4 on a context whose keys are set: the saturated capacity from a
    burst of `burst` requests, then `per_rate` requests as a Poisson stream at
    0.3, 0.6 and 0.9 of it; requests drawn uniformly from `table`, admission
    by free device memory (the ciphertext pool grows from free HBM), gates
    batched across requests per level.  Every add32 and mul32 result is
    checked by decryption.  -> (capacity dict, per-rate list)."""
    import torch
    from paper_2005_01945_gb300 import api, synth
    variants = 8
    inputs = {}   # per kind: (A, B, plaintexts) with `variants` distinct operands
    for name, kind, w in table:
        a, b = synth.int_pairs(variants, w, seed, name)
        ba, bb = synth.to_bits(a, w), synth.to_bits(b, w)
        ca = synth.ct_draws(p, ba.shape, seed, name + "a")
        cb = synth.ct_draws(p, bb.shape, seed, name + "b")
        inputs[name] = (api.encrypt_bits(p, s_dev, d(ca.mask), d(ca.noise), d(ba)),
                        api.encrypt_bits(p, s_dev, d(cb.mask), d(cb.noise), d(bb)), a, b)
    gates_of = {name: (1 if kind == 0 else api.circuit_info(kind, w)[0])
                for name, kind, w in table}
    dev = s_dev.device

    def run_stream(arrivals, kinds, budget=0):   # 0: the pool grows from free HBM
        outs = {name: torch.empty((max(1, int((kinds == k).sum())), w, api.LWE_STRIDE),
                                  dtype=torch.int32, device=dev)
                for k, (name, kind, w) in enumerate(table)}
        used = {name: 0 for name, _, _ in table}
        ctx.serve_start(budget)
        ids, meta = [], []
        t0 = time.perf_counter()
        for t_arr, k in zip(arrivals, kinds):
            name, kind, w = table[k]
            while time.perf_counter() - t0 < t_arr:
                time.sleep(0.0002)
            A, B, _, _ = inputs[name]
            v = len(ids) % variants
            slot = used[name]
            used[name] += 1
            out = outs[name][slot]
            width = 3 if kind == 0 else w          # a single gate is an XOR
            ids.append(ctx.serve_submit(kind, width, A[v], B[v], out))
            meta.append((name, v, slot))
        lats = np.array([ctx.serve_wait(i, 600000) for i in ids])
        stats = ctx.serve_stats()
        ctx.serve_stop()
        torch.cuda.synchronize()
        # verify the multiplications and additions of the stream by decryption
        ok = True
        for name in ("mul32", "add32"):
            _, _, a, b = inputs[name]
            w = 32
            k = used[name]
            if k == 0:
                continue
            dec = synth.from_bits(api.decrypt_bits(p, s_dev, outs[name][:k]).cpu().numpy())
            vs = np.array([v for (nm, v, _) in meta if nm == name])
            want = (a[vs] * b[vs] if name == "mul32" else a[vs] + b[vs]) % (1 << w)
            ok &= bool(np.array_equal(dec, want))
        wall = stats["wall_ms"] / 1e3
        return lats, stats, wall, ok, [m[0] for m in meta]

    # saturated capacity: a burst of requests all at once
    rng = np.random.default_rng(seed)
    kinds = rng.integers(0, len(table), size=burst)
    _, stats, wall, ok_cap, _ = run_stream(np.zeros(burst), kinds)
    cap_gates = stats["gates"] / wall
    mean_gates = float(np.mean([gates_of[n] for n, _, _ in table]))
    cap_req = cap_gates / mean_gates
    capacity = {"burst_requests": burst, "gates_per_s": cap_gates, "req_per_s": cap_req,
                "mean_gates_per_request": mean_gates, "verified": ok_cap}
    results = []
    for frac in (0.3, 0.6, 0.9):
        lam = frac * cap_req
        arr = np.cumsum(rng.exponential(1.0 / lam, size=per_rate))
        kinds = rng.integers(0, len(table), size=per_rate)
        lats, stats, wall, ok, names = run_stream(arr, kinds)
        names = np.array(names)
        m32 = lats[names == "mul32"]
        results.append({"load": frac, "offered_req_per_s": lam, "requests": per_rate,
                        "gates_per_s": stats["gates"] / wall, "iterations": stats["iterations"],
                        "admitted_while_others_ran": stats["admitted_busy"],
                        "pool_bytes": stats["pool_bytes"], "pool_grows": stats["pool_grows"],
                        "p50_ms": float(np.percentile(lats, 50)),
                        "p99_ms": float(np.percentile(lats, 99)),
                        "mul32_p50_ms": float(np.percentile(m32, 50)) if len(m32) else None,
                        "mul32_p99_ms": float(np.percentile(m32, 99)) if len(m32) else None,
                        "verified": ok})
    return capacity, results


def run_serve(args):
    """Config 4: a Poisson request stream at 0.3, 0.6 and 0.9 of the measured
    saturated request rate, requests drawn uniformly from {single gate,
    16-bit add, 32-bit add, 16-bit mul, 32-bit mul}; keys device-resident,
    admission by free device memory (the ciphertext pool grows from free HBM),
    gates batched across requests per level."""
    from paper_2005_01945_gb300 import api, build, synth
    build.build()
    table = SERVE_KINDS_SHALLOW if args.serve_circuits == "shallow" else SERVE_KINDS
    p = synth.TFHEParams()
    seed = synth.MASTER_SEED + 4
    kd = synth.key_draws(p, seed)
    d = api.to_device
    bk, ksk = api.keygen(p, d(kd.s), d(kd.S), d(kd.bk_mask), d(kd.bk_noise), d(kd.ksk_mask),
                         d(kd.ksk_noise))
    ctx = api.Context(p)
    ctx.set_keys(bk, ksk)
    # launch shapes and the level times the serving loop's iteration choice uses
    ctx.autotune(args.tune_cache)
    capacity, results = measure_serving(ctx, p, d(kd.s), d, seed, table,
                                        args.serve_requests // 3)
    print(json.dumps({"metric": "serving: p50/p99 request latency and gates/s under Poisson load",
                      "config": {"workload": "config 4: requests uniform over {XOR gate, add16, "
                                             "add32, mul16, mul32}; mean "
                                             f"{capacity['mean_gates_per_request']:.1f} "
                                             "gates/request",
                                 "circuits": args.serve_circuits,
                                 "capacity_gates_per_s": capacity["gates_per_s"],
                                 "capacity_req_per_s": capacity["req_per_s"]},
                      "rates": results}), flush=True)
    ctx.close()


def br_roofline(p, br_ms, br_launch, br_boot, step_ms_total, ks_ms, sm_count, sm_max):
    """Roofline of the blind-rotation kernel from the CUDA events recorded
    around its launches: algorithmic INT32 operations / device time, against
    SMs x 128 INT32 lanes x clock."""
    peak_ops = sm_count * INT32_LANES_PER_SM * sm_max * 1e6
    ops = OPS_PER_CMUX * p.n * br_boot
    achieved = ops / (br_ms / 1e3) if br_ms > 0 else 0.0
    return {"kernel": "k_blind_rotate", "bound": "alu", "achieved": achieved / 1e12,
            "peak": peak_ops / 1e12, "unit": "Tops/s (int32)", "frac": achieved / peak_ops,
            "peak_basis": f"{sm_count} SMs x {INT32_LANES_PER_SM} INT32 "
                          f"lanes x {sm_max:.0f} MHz (max SM clock)",
            "launches": br_launch, "bootstraps": br_boot,
            "avg_launch_ms": br_ms / max(br_launch, 1),
            "share_of_step": br_ms / max(step_ms_total, 1e-9),
            "keyswitch_share_of_step": ks_ms / max(step_ms_total, 1e-9)}


def run_config_steps(ctx, fn, steps, flush, e0, e1):
    """One warm-up run, then `steps` timed runs (L2 flushed before each) with
    the blind-rotation / key-switch events of every run summed."""
    import torch
    fn()
    torch.cuda.synchronize()
    ctx.profile()
    ms, br_ms, br_l, br_b, ks_ms = [], 0.0, 0, 0, 0.0
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        pr = ctx.profile()
        br_ms += pr["br_ms"]
        br_l += pr["br_launches"]
        br_b += pr["br_bootstraps"]
        ks_ms += pr["ks_ms"]
    return ms, br_ms, br_l, br_b, ks_ms


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.br_only:
        run_br_only(args.br_only, args.br_group)
        return
    if args.ks_only:
        run_ks_only(args.ks_only, args.ks_kernel)
        return
    if args.tc_products:
        run_tc_products(args.tc_products)
        return
    if args.serve:
        run_serve(args)
        return
    if args.configs:
        run_configs(args)
        return
    if args.variants:
        run_variants(args)
        return
    import torch
    from paper_2005_01945_gb300 import api, build, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    dev = torch.device("cuda", local)

    # ---- keys and inputs (synthetic, seeded; every rank its own replica)
    seed = synth.MASTER_SEED + 1000 * rank
    p = synth.TFHEParams()
    kd = synth.key_draws(p, seed)
    d = lambda a: api.to_device(a, dev)  # noqa: E731
    bk, ksk = api.keygen(p, d(kd.s), d(kd.S), d(kd.bk_mask), d(kd.bk_noise), d(kd.ksk_mask),
                         d(kd.ksk_noise))
    ctx = api.Context(p, device=local)
    ctx.set_keys(bk, ksk)
    del bk, ksk
    s_dev = d(kd.s)
    a, b = synth.int_pairs(BATCH, WIDTH, seed + 1, "add32")
    ba, bb = synth.to_bits(a, WIDTH), synth.to_bits(b, WIDTH)
    cda = synth.ct_draws(p, ba.shape, seed + 1, "add32a")
    cdb = synth.ct_draws(p, bb.shape, seed + 1, "add32b")
    A = api.encrypt_bits(p, s_dev, d(cda.mask), d(cda.noise), d(ba))
    B = api.encrypt_bits(p, s_dev, d(cdb.mask), d(cdb.noise), d(bb))
    R = torch.empty_like(A)
    gates_step = BATCH * GATES_PER_ADD
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def barrier():
        if dist is not None:
            dist.barrier()

    tuned = ctx.autotune(args.tune_cache)
    ctx.set_option(api.OPT_PROFILE, 1)
    for _ in range(args.warmup):
        ctx.add_n(WIDTH, A, B, R)
    torch.cuda.synchronize()
    ctx.profile()

    # ---- timed region: K steps, L2 flushed between steps
    sampler = ClockSampler(local)
    sampler.start()
    step_ms, br_ms, br_launch, br_boot, ks_ms = [], 0.0, 0, 0, 0.0
    launches0 = ctx.launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        e0.record()
        ctx.add_n(WIDTH, A, B, R)
        e1.record()
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        pr = ctx.profile()
        br_ms += pr["br_ms"]
        br_launch += pr["br_launches"]
        br_boot += pr["br_bootstraps"]
        ks_ms += pr["ks_ms"]
    barrier()
    launches = ctx.launches() - launches0
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    value = whole_job_rate(gates_step, args.steps, world, total_ms)

    # ---- correctness of the timed result (decryption on the device)
    dec = api.decrypt_bits(p, s_dev, R).cpu().numpy()
    verified = bool(np.array_equal(synth.from_bits(dec), (a + b) % (1 << WIDTH)))

    # ---- end to end: pinned host ciphertexts in, results out, every step
    ctx.set_option(api.OPT_PROFILE, 0)
    A_h = A.cpu().pin_memory()
    B_h = B.cpu().pin_memory()
    R_h = torch.empty(R.shape, dtype=R.dtype).pin_memory()
    ctx.add_n(WIDTH, A, B, R)
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        e0.record()
        A.copy_(A_h, non_blocking=True)
        B.copy_(B_h, non_blocking=True)
        ctx.add_n(WIDTH, A, B, R)
        R_h.copy_(R, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_total = max_over_ranks(sum(e2e_ms), dist, dev)
    e2e = {"value": whole_job_rate(gates_step, args.steps, world, e2e_total), "unit": "gates/s",
           "h2d_bytes_per_step": A.numel() * 4 + B.numel() * 4,
           "d2h_bytes_per_step": R.numel() * 4}

    # ---- roofline of the dominant kernel (blind rotation), from the events
    # recorded around its launches inside the timed graph replays
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = props.multi_processor_count
    roofline = br_roofline(p, br_ms, br_launch, br_boot, sum(step_ms), ks_ms, nsm, sm_max)
    roofline.update({"traffic": br_traffic_per_launch(),
                     "traffic_unit": "bytes per launch (ncu dram)",
                     "algorithmic_bytes_per_launch": 32.8e6 + br_boot / max(br_launch, 1) * 8192})
    # key switch (one call per level: the tiled kernel and its output
    # initialisation), against HBM: algorithmic bytes = the key once + the
    # level's LWE_N inputs and LWE_n outputs
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    ks_calls = max(br_launch, 1)
    ks_bytes = KSK_BYTES + br_boot / ks_calls * (p.N + 1 + p.n + 1) * 4
    ks_gbs = ks_bytes / (ks_ms / ks_calls / 1e3) / 1e9 if ks_ms > 0 else 0.0
    keyswitch = {"kernel": "k_keyswitch_tiled", "bound": "smem", "achieved_hbm": ks_gbs,
                 "peak_hbm": hbm, "unit": "GB/s", "frac_hbm": ks_gbs / hbm,
                 "algorithmic_bytes_per_call": ks_bytes, "calls": ks_calls,
                 "avg_call_ms": ks_ms / ks_calls,
                 "note": "reads the key once per call from DRAM; bound by shared-memory "
                         "bandwidth (selected key rows delivered per gate), not HBM"}

    # ---- configs 2 and 3 (device-resident inputs, L2 flushed before each
    # timed run, same keys and tuned shapes), each verified by decryption
    configs = None
    if rank == 0 and args.config_steps > 0:
        ctx.set_option(api.OPT_PROFILE, 1)

        def enc(xs, w, s_, tag):
            bits = synth.to_bits(xs, w)
            cd = synth.ct_draws(p, bits.shape, s_, tag)
            return api.encrypt_bits(p, s_dev, d(cd.mask), d(cd.noise), d(bits))

        dec = lambda t: synth.from_bits(api.decrypt_bits(p, s_dev, t).cpu().numpy())  # noqa: E731
        configs = {}
        a16, b16 = synth.int_pairs(64, 16, seed + 2, "mul16")
        a32, b32 = synth.int_pairs(64, 32, seed + 2, "mul32")
        A16, B16 = enc(a16, 16, seed + 2, "m16a"), enc(b16, 16, seed + 2, "m16b")
        A32, B32 = enc(a32, 32, seed + 2, "m32a"), enc(b32, 32, seed + 2, "m32b")
        R16, R32 = torch.empty_like(A16), torch.empty_like(A32)
        jobs = [dict(kind=api.MUL, width=16, batch=64, in0=A16, in1=B16, out=R16),
                dict(kind=api.MUL, width=32, batch=64, in0=A32, in1=B32, out=R32)]
        M = synth.random_uints((16, 16), 16, seed + 3, "M")
        v = synth.random_uints(16, 16, seed + 3, "v")
        MM, vv = enc(M, 16, seed + 3, "M"), enc(v, 16, seed + 3, "v")
        y = torch.empty((16, 16, api.LWE_STRIDE), dtype=torch.int32, device=dev)
        work = [
            ("config2_mul16x64_mul32x64",
             "64 16-bit and 64 32-bit shift-and-add multiplications (truncated) of uniform "
             "random operands in one level schedule (depths 56 and 120)",
             lambda: ctx.run_jobs(jobs),
             64 * (api.circuit_info(api.MUL, 16)[0] + api.circuit_info(api.MUL, 32)[0]),
             lambda: bool(np.array_equal(dec(R16), (a16 * b16) % (1 << 16)) and
                          np.array_equal(dec(R32), (a32 * b32) % (1 << 32)))),
            ("config3_matvec16x16",
             "16x16 matrix of uniform uint16 times a uint16 vector, products by shift-and-add "
             "multipliers, row sums by a tree of 16-bit ripple-carry adders (mod 2^16)",
             lambda: ctx.matvec(16, MM, vv, y),
             api.circuit_info(api.MATVEC, 16, 16, 16)[0],
             lambda: bool(np.array_equal(dec(y), (M * v[None, :]).sum(axis=1) % (1 << 16)))),
        ]
        for name, desc, fn, gates, check in work:
            ms, cbr, cbl, cbb, cks = run_config_steps(ctx, fn, args.config_steps, flush, e0, e1)
            rl = br_roofline(p, cbr, cbl, cbb, sum(ms), cks, nsm, sm_max)
            configs[name] = {"workload": desc, "gates_per_step": gates,
                             "steps": len(ms), "warmup": 1, "ms_per_step": float(np.mean(ms)),
                             "gates_per_s": gates * len(ms) / (sum(ms) / 1e3),
                             "levels_per_step": cbl // max(len(ms), 1),
                             "bootstraps_per_launch": cbb / max(cbl, 1),
                             "roofline": {k: rl[k] for k in ("kernel", "bound", "achieved",
                                                             "peak", "unit", "frac",
                                                             "avg_launch_ms", "launches",
                                                             "share_of_step",
                                                             "keyswitch_share_of_step")},
                             "verified": check()}
        ctx.set_option(api.OPT_PROFILE, 0)

    # ---- 32-bit multiplication latency: level-batched vs one launch pair per
    # gate, for the sequential shift-and-add multiplier and for the
    # Dadda-tree multiplier
    latency = latency_tree = None
    if not args.no_latency and rank == 0:
        ma, mb = synth.int_pairs(1, 32, seed + 2, "lat")
        da = api.encrypt_bits(p, s_dev, d(synth.ct_draws(p, (1, 32), seed + 2, "la").mask),
                              d(synth.ct_draws(p, (1, 32), seed + 2, "la").noise),
                              d(synth.to_bits(ma, 32)))
        db = api.encrypt_bits(p, s_dev, d(synth.ct_draws(p, (1, 32), seed + 2, "lb").mask),
                              d(synth.ct_draws(p, (1, 32), seed + 2, "lb").noise),
                              d(synth.to_bits(mb, 32)))
        out = torch.empty((1, 32, api.LWE_STRIDE), dtype=torch.int32, device=dev)
        want = (int(ma[0]) * int(mb[0])) % (1 << 32)

        def measure(kind, per_gate_samples):
            job = [dict(kind=kind, width=32, batch=1, in0=da, in1=db, out=out)]

            def timed(nsamp):
                res = []
                ctx.run_jobs(job)
                torch.cuda.synchronize()
                for _ in range(nsamp):
                    e0.record()
                    ctx.run_jobs(job)
                    e1.record()
                    torch.cuda.synchronize()
                    res.append(e0.elapsed_time(e1))
                return res

            ok = lambda: bool(synth.from_bits(api.decrypt_bits(p, s_dev, out).cpu().numpy())[0]  # noqa: E731
                              == want)
            batched = timed(args.latency_samples)
            ok_b = ok()
            ctx.set_option(api.OPT_PER_GATE, 1)
            per_gate = timed(per_gate_samples)
            ctx.set_option(api.OPT_PER_GATE, 0)
            ok_p = ok()
            gates, depth = api.circuit_info(kind, 32)
            pct = lambda xs, q: float(np.percentile(np.array(xs), q))  # noqa: E731
            res = {"gates": gates, "levels": depth,
                   "batched_p50_ms": pct(batched, 50), "batched_p99_ms": pct(batched, 99),
                   "batched_samples": len(batched),
                   "per_gate_p50_ms": pct(per_gate, 50), "per_gate_max_ms": max(per_gate),
                   "per_gate_samples": len(per_gate), "verified": ok_b and ok_p}
            # a 99th percentile needs enough samples to differ from the maximum
            if len(per_gate) >= 10:
                res["per_gate_p99_ms"] = pct(per_gate, 99)
            return res

        latency = measure(api.MUL, args.per_gate_samples)
        latency["request"] = ("one 32x32->32 sequential shift-and-add multiplication "
                              "(2,824 gates, 120 levels) alone")
        latency_tree = measure(api.MUL_DADDA, args.per_gate_samples_shallow)
        latency_tree["request"] = ("one 32x32->32 multiplication, partial products reduced by a "
                                   "Dadda tree of full adders (majority carries) and summed by a "
                                   f"parallel-prefix adder ({latency_tree['gates']:,} gates, "
                                   f"{latency_tree['levels']} levels) alone")

    # ---- the exact-product choice: tensor-pipe CMux products vs the NTT CMux
    product_choice = None
    if rank == 0 and args.product_choice > 0:
        product_choice = tc_vs_ntt(ctx, p, kd, args.product_choice, device=dev)
        product_choice = {k: v for k, v in product_choice.items()
                          if k not in ("tc_prepare_key_ms", "tc_products_ms", "ntt_blind_rotation_ms")}

    # ---- config 4 (bounded): serving capacity and a Poisson stream of
    # args.serve_sample requests at each of 0.3, 0.6 and 0.9 of it, same keys
    # and tuned shapes; `python bench.py --serve` runs the 10,000-request form
    serving = None
    if rank == 0 and args.serve_sample > 0:
        capacity, rates = measure_serving(ctx, p, s_dev, d, seed + 4, SERVE_KINDS,
                                          args.serve_sample)
        serving = {"workload": "config 4: requests uniform over {XOR gate, add16, add32, "
                               "mul16, mul32} (ripple-carry adders, shift-and-add "
                               "multipliers), admission by free HBM",
                   "requests_per_rate": args.serve_sample, "capacity": capacity,
                   "rates": rates}

    cpu = None
    if rank == 0 and world == 1 and args.cpu_gates > 0:
        sample = OracleSample(args.cpu_gates, seed)
        rate = sample.rate()
        cpu = {"value": rate, "unit": "gates/s", "cores": sample.cores, "kind": "oracle",
               "sample": sample.desc}
        if args.cpu_gates_single > 0:
            one = sample.rate(args.cpu_gates_single, threads=1)
            cpu["single_thread"] = {"value": one, "unit": "gates/s", "cores": 1,
                                    "sample": f"the first {min(args.cpu_gates_single, args.cpu_gates)} "
                                              "gates of the same sample on one thread"}
        g3 = 16 * 16 * 648 + 16 * 15 * 74
        cpu["config3_extrapolated"] = {
            "gates": g3, "seconds_all_cores": g3 / rate,
            "seconds_one_thread": g3 / cpu["single_thread"]["value"] if "single_thread" in cpu
            else None,
            "basis": "extrapolated, not run: the 16x16 matvec's gate count divided by the "
                     "oracle's measured gate rate on the sample (every gate is one bootstrap + "
                     "key switch of the same cost; the oracle's circuit evaluation keeps all "
                     "cores busy on this workload's 256 independent products)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "gates/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "gates_per_step": gates_step, "batch": BATCH,
                           "width": WIDTH, "levels": 62,
                           "l2": "flushed between timed steps (256 MB write)",
                           "schedule": "deadline-balanced levels, one wave (4 bootstraps/SM)",
                           "autotuned": tuned,
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
                "keyswitch": keyswitch,
                "cpu_baseline": cpu, "configs": configs, "product_choice": product_choice,
                "mul32_latency": latency,
                "mul32_shallow_latency": latency_tree, "serving": serving,
                "verified": verified}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
