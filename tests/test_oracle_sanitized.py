"""The oracle under the undefined-behaviour sanitizer.

The oracle is plain C whose exactness rests on unsigned 32-bit wraparound
and on 64-bit intermediates in its rounding; a signed overflow, an
over-wide shift or an out-of-range index would be undefined behaviour that
an optimising compiler may turn into a silently different result.  This
test compiles a second copy of the oracle with -fsanitize=undefined (abort
on the first report), runs every kind of oracle call on toy parameters in a
child process against it, and checks that the child exits cleanly and
computes exactly what the normal -O3 build computes."""
import hashlib
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# One script, run in this process against the normal build and in a child
# against the sanitized one; it prints a digest of every output.
SCRIPT = textwrap.dedent("""
    import hashlib, sys
    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle
    if LIB:
        oracle._LIB, oracle._lib = LIB, None
        oracle.build = lambda force=False: LIB
    from paper_2005_01945_gb300 import synth
    h = hashlib.sha256()
    def put(a):
        h.update(np.ascontiguousarray(a).tobytes())
    rng = np.random.default_rng(7)
    for N in (4, 16, 64):
        a = rng.integers(0, 2**32, N, dtype=np.uint64).astype(np.uint32)
        b = rng.integers(0, 2**32, N, dtype=np.uint64).astype(np.uint32)
        put(oracle.negacyclic_mul(a, b))
        for k in (0, 1, N - 1, N, 2 * N - 1):
            put(oracle.mul_by_xk(a, k))
    x = rng.integers(0, 2**32, 4096, dtype=np.uint64).astype(np.uint32)
    x[:6] = [0, 1, 2**31 - 1, 2**31, 2**32 - 1, 2**21]
    put(oracle.decompose(x, 10, 2))
    put(oracle.modswitch(x, 1024))
    p = synth.TFHEParams(n=8, N=32)
    P = oracle.Params(p.n, p.N, p.l, p.bg_bit, p.ks_t, p.ks_basebit)
    kd = synth.key_draws(p, 5)
    bk = oracle.keygen_bk(P, kd.s, kd.S, kd.bk_mask, kd.bk_noise)
    ksk = oracle.keygen_ksk(P, kd.s, kd.S, kd.ksk_mask, kd.ksk_noise)
    put(bk); put(ksk)
    def enc(xs, w, tag):
        bits = synth.to_bits(xs, w)
        cd = synth.ct_draws(p, bits.shape, 5, tag)
        return oracle.encrypt_bits(P, kd.s, cd.mask, cd.noise, bits)
    g = 12
    ops = (np.arange(g) % 6).astype(np.uint8)
    ca, cb = enc(np.arange(g) & 1, 1, "ga")[:, 0], enc(np.arange(g) >> 1 & 1, 1, "gb")[:, 0]
    put(oracle.gates(P, bk, ksk, ops, ca, cb))
    put(oracle.gate3(P, bk, ksk, 6, ca[:4], cb[:4], ca[4:8]))
    A = enc(np.array([3, 250, 0, 255]), 8, "A")
    B = enc(np.array([7, 9, 255, 255]), 8, "B")
    for f in (oracle.add, oracle.mul, oracle.add_maj, oracle.add_nw, oracle.add_prefix,
              oracle.mul_tree, oracle.mul_tree_maj, oracle.mul_dadda, oracle.mul_full,
              oracle.mul_karatsuba):
        r = f(P, bk, ksk, 8, A, B)
        put(r[0] if isinstance(r, tuple) else r)
    M = enc(np.array([[1, 2, 3], [4, 5, 6]]), 4, "M")
    v = enc(np.array([7, 8, 9]), 4, "v")
    r = oracle.matvec(P, bk, ksk, 4, M, v)
    put(r[0] if isinstance(r, tuple) else r)
    print(h.hexdigest())
""")


def _digest(lib_path):
    code = f"ROOT = {ROOT!r}\nLIB = {lib_path!r}\n" + SCRIPT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       timeout=600, env=dict(os.environ, OMP_NUM_THREADS="4"))
    return r


def test_oracle_has_no_undefined_behaviour(tmp_path, orc):
    lib = str(tmp_path / "libtfhe_oracle_ubsan.so")
    cmd = ["gcc", "-O1", "-g", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-fsanitize=undefined", "-fno-sanitize-recover=all", "-static-libubsan",
           os.path.join(ROOT, "oracle", "tfhe_oracle.c"), "-o", lib]
    if subprocess.run(cmd, capture_output=True).returncode != 0:
        pytest.skip("gcc cannot build a sanitized shared library here")
    plain = _digest("")
    assert plain.returncode == 0, plain.stderr[-2000:]
    checked = _digest(lib)
    assert checked.returncode == 0, checked.stderr[-2000:]
    assert "runtime error" not in checked.stderr, checked.stderr[-2000:]
    assert checked.stdout.strip() == plain.stdout.strip()
    assert len(plain.stdout.strip()) == 64
