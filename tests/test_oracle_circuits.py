"""Pins for the oracle's circuits: decryption equals the plaintext result
on every output (add, mul mod 2^w; matrix-vector product mod 2^w), and the
bootstrapped-gate counts equal the counts of the circuit definitions."""
import os

import numpy as np
import pytest

from conftest import oparams, toy_params
from paper_2005_01945_gb300 import synth


def _counts():
    path = os.path.join(os.path.dirname(__file__), "golden", "circuit_gate_counts.txt")
    out = {}
    for line in open(path):
        f = line.split("#")[0].split()
        if len(f) == 5:
            out[(f[0], int(f[1]), int(f[2]), int(f[3]))] = int(f[4])
    return out


@pytest.fixture(scope="module")
def toy(orc):
    p = toy_params(n=8, N=32)
    P = oparams(p)
    kd = synth.key_draws(p, 31)
    bk = orc.keygen_bk(P, kd.s, kd.S, kd.bk_mask, kd.bk_noise)
    ksk = orc.keygen_ksk(P, kd.s, kd.S, kd.ksk_mask, kd.ksk_noise)
    return p, P, kd, bk, ksk


def _enc_ints(orc, p, P, kd, xs, w, tag):
    bits = synth.to_bits(xs, w)
    cd = synth.ct_draws(p, bits.shape, 77, tag)
    return orc.encrypt_bits(P, kd.s, cd.mask, cd.noise, bits)


def _dec_ints(orc, P, kd, cts):
    return synth.from_bits(orc.decrypt_bits(P, kd.s, cts))


@pytest.mark.parametrize("w", [1, 2, 3, 4])
def test_add_exhaustive(orc, toy, w):
    p, P, kd, bk, ksk = toy
    a, b = np.meshgrid(np.arange(1 << w), np.arange(1 << w), indexing="ij")
    a, b = a.ravel().astype(np.uint64), b.ravel().astype(np.uint64)
    R, g = orc.add(P, bk, ksk, w, _enc_ints(orc, p, P, kd, a, w, f"a{w}"),
                   _enc_ints(orc, p, P, kd, b, w, f"b{w}"))
    assert np.array_equal(_dec_ints(orc, P, kd, R), (a + b) % (1 << w))
    key = ("add", w, 0, 0)
    if key in _counts():
        assert g == len(a) * _counts()[key]


@pytest.mark.parametrize("w", [8, 16, 32])
def test_add_random_wide(orc, toy, w):
    p, P, kd, bk, ksk = toy
    a, b = synth.int_pairs(16, w, 5, f"add{w}")
    R, g = orc.add(P, bk, ksk, w, _enc_ints(orc, p, P, kd, a, w, "wa"),
                   _enc_ints(orc, p, P, kd, b, w, "wb"))
    assert np.array_equal(_dec_ints(orc, P, kd, R), (a + b) % (1 << w))
    assert g == 16 * (5 * w - 6)


@pytest.mark.parametrize("w", [1, 2, 3, 4])
def test_mul_exhaustive(orc, toy, w):
    p, P, kd, bk, ksk = toy
    a, b = np.meshgrid(np.arange(1 << w), np.arange(1 << w), indexing="ij")
    a, b = a.ravel().astype(np.uint64), b.ravel().astype(np.uint64)
    R, g = orc.mul(P, bk, ksk, w, _enc_ints(orc, p, P, kd, a, w, f"ma{w}"),
                   _enc_ints(orc, p, P, kd, b, w, f"mb{w}"))
    assert np.array_equal(_dec_ints(orc, P, kd, R), (a * b) % (1 << w))
    key = ("mul", w, 0, 0)
    if key in _counts():
        assert g == len(a) * _counts()[key]


@pytest.mark.parametrize("w", [16, 32])
def test_mul_gate_counts_and_values(orc, toy, w):
    p, P, kd, bk, ksk = toy
    a, b = synth.int_pairs(2, w, 6, f"mul{w}")
    R, g = orc.mul(P, bk, ksk, w, _enc_ints(orc, p, P, kd, a, w, "xa"),
                   _enc_ints(orc, p, P, kd, b, w, "xb"))
    assert np.array_equal(_dec_ints(orc, P, kd, R), (a * b) % (1 << w))
    assert g == 2 * _counts()[("mul", w, 0, 0)]


def test_matvec_odd_tree(orc, toy):
    """3 x 5 matrix (an odd number of terms per row exercises the tree's
    carried element), 4-bit entries."""
    p, P, kd, bk, ksk = toy
    w, rows, cols = 4, 3, 5
    M = synth.random_uints((rows, cols), w, 8, "M")
    v = synth.random_uints(cols, w, 8, "v")
    Y, g = orc.matvec(P, bk, ksk, w, _enc_ints(orc, p, P, kd, M, w, "M"),
                      _enc_ints(orc, p, P, kd, v, w, "v"))
    want = (M.astype(np.uint64) * v[None, :]).sum(axis=1) % (1 << w)
    assert np.array_equal(_dec_ints(orc, P, kd, Y), want)
    assert g == _counts()[("matvec", w, rows, cols)]


def test_count_table_consistent():
    """The stored counts agree with each other through their recurrences."""
    c = _counts()
    add = lambda w: 1 if w == 1 else 5 * w - 6
    mul = lambda w: w * (w + 1) // 2 + sum(add(m) for m in range(1, w))
    for (kind, w, r, k), g in c.items():
        if kind == "add":
            assert g == add(w)
        elif kind == "mul":
            assert g == mul(w)
        else:
            assert g == r * (k * mul(w) + (k - 1) * add(w))


def test_library_netlists_match_count_table():
    """The CUDA library's netlist builder (host code, no GPU needed) has the
    gate counts of the circuit definitions, and the 32-bit adder's ASAP
    depth is 2 (first XOR/AND level) + 2 per middle bit = 62."""
    from paper_2005_01945_gb300 import api, build
    build.build()
    kinds = {"add": api.ADD, "mul": api.MUL, "matvec": api.MATVEC}
    for (kind, w, r, c), g in _counts().items():
        assert api.circuit_info(kinds[kind], w, r, c)[0] == g
    assert api.circuit_info(api.ADD, 32)[1] == 62


def test_balanced_schedule_invariants():
    """Host-only schedules: the deadline-driven list schedule keeps the ASAP
    depth, covers every gate once, and keeps levels at the target width
    wherever deadlines allow (for the 256 x add32 batch: all but the last)."""
    from paper_2005_01945_gb300 import api, build
    build.build()
    for jobs in ([(api.ADD, 32, 0, 0, 256)], [(api.MUL, 16, 0, 0, 64), (api.MUL, 32, 0, 0, 64)],
                 [(api.MATVEC, 8, 4, 5, 2)], [(api.GATE, api.XOR, 0, 0, 100)]):
        wa, ga = api.schedule_info(jobs, api.SCHED_ASAP, 608)
        wb, gb = api.schedule_info(jobs, api.SCHED_BALANCED, 608)
        assert ga == gb == sum(k[4] * api.circuit_info(k[0], k[1], k[2], k[3])[0] for k in jobs)
        assert wa.sum() == wb.sum() == ga
        assert len(wb) == len(wa)
        assert wb.min() > 0
    wb, _ = api.schedule_info([(api.ADD, 32, 0, 0, 256)], api.SCHED_BALANCED, 608)
    assert (wb[:-1] == 608).all() and wb[-1] == 39424 - 61 * 608


@pytest.mark.parametrize("name", ["add_maj", "add_nw", "mul_tree", "mul_tree_maj", "add_prefix",
                                  "mul_dadda"])
@pytest.mark.parametrize("w", [1, 2, 3, 4])
def test_new_circuits_exhaustive(orc, toy, name, w):
    """Majority-carry adder, the paper's number-wise adder GPU_n,
    tree-accumulated multiplication (ripple or majority carries), the
    parallel-prefix adder and the Dadda multiplier: every input pair at toy
    parameters."""
    p, P, kd, bk, ksk = toy
    a, b = np.meshgrid(np.arange(1 << w), np.arange(1 << w), indexing="ij")
    a, b = a.ravel().astype(np.uint64), b.ravel().astype(np.uint64)
    R, g = getattr(orc, name)(P, bk, ksk, w, _enc_ints(orc, p, P, kd, a, w, f"{name}a{w}"),
                              _enc_ints(orc, p, P, kd, b, w, f"{name}b{w}"))
    want = (a * b if name.startswith("mul") else a + b) % (1 << w)
    assert np.array_equal(_dec_ints(orc, P, kd, R), want)


@pytest.mark.parametrize("w", [5, 6])
def test_prefix_adder_and_dadda_exhaustive_w5_w6(orc, toy, w):
    """Parallel-prefix adder and Dadda multiplier at widths where the prefix
    network has 3 and 3 levels with ragged blocks (w - 1 = 4, 5) and the
    Dadda tree 2 and 3 stages: every input pair at toy parameters."""
    p, P, kd, bk, ksk = toy
    a, b = np.meshgrid(np.arange(1 << w), np.arange(1 << w), indexing="ij")
    a, b = a.ravel().astype(np.uint64), b.ravel().astype(np.uint64)
    A = _enc_ints(orc, p, P, kd, a, w, f"pxa{w}")
    B = _enc_ints(orc, p, P, kd, b, w, f"pxb{w}")
    R, _ = orc.add_prefix(P, bk, ksk, w, A, B)
    assert np.array_equal(_dec_ints(orc, P, kd, R), (a + b) % (1 << w))
    R, _ = orc.mul_dadda(P, bk, ksk, w, A, B)
    assert np.array_equal(_dec_ints(orc, P, kd, R), (a * b) % (1 << w))


@pytest.mark.parametrize("w", [8, 16, 32])
def test_new_circuits_wide_and_counts(orc, toy, w):
    """Random wide operands; gate counts: majority adder 3w - 2, number-wise
    adder w^2, and the oracle's counts equal the CUDA library's netlists
    (two independent implementations of the circuit definitions)."""
    from paper_2005_01945_gb300 import api, build
    build.build()
    p, P, kd, bk, ksk = toy
    a, b = synth.int_pairs(3, w, 9, f"nc{w}")
    A, B = _enc_ints(orc, p, P, kd, a, w, "nca"), _enc_ints(orc, p, P, kd, b, w, "ncb")
    for name, kind, want in (("add_maj", api.ADD_MAJ, (a + b) % (1 << w)),
                             ("add_nw", api.ADD_NW, (a + b) % (1 << w)),
                             ("mul_tree", api.MUL_TREE, (a * b) % (1 << w)),
                             ("mul_tree_maj", api.MUL_TREE_MAJ, (a * b) % (1 << w)),
                             ("add_prefix", api.ADD_PREFIX, (a + b) % (1 << w)),
                             ("mul_dadda", api.MUL_DADDA, (a * b) % (1 << w))):
        R, g = getattr(orc, name)(P, bk, ksk, w, A, B)
        assert np.array_equal(_dec_ints(orc, P, kd, R), want), name
        assert g == 3 * api.circuit_info(kind, w)[0], name
    assert api.circuit_info(api.ADD_MAJ, w) == (3 * w - 2, w)
    assert api.circuit_info(api.ADD_NW, w) == (w * w, w)


@pytest.mark.parametrize("w", [2, 3, 4])
def test_full_products_exhaustive(orc, toy, w):
    """Full products (2w bits): the naive product and Karatsuba (which is
    the naive product below its 8-bit base case) on every input pair."""
    p, P, kd, bk, ksk = toy
    a, b = np.meshgrid(np.arange(1 << w), np.arange(1 << w), indexing="ij")
    a, b = a.ravel().astype(np.uint64), b.ravel().astype(np.uint64)
    A = _enc_ints(orc, p, P, kd, a, w, f"fpa{w}")
    B = _enc_ints(orc, p, P, kd, b, w, f"fpb{w}")
    for name in ("mul_full", "mul_karatsuba"):
        R, g = getattr(orc, name)(P, bk, ksk, w, A, B)
        assert R.shape == (len(a), 2 * w, P.n + 1)
        assert np.array_equal(_dec_ints(orc, P, kd, R), a * b), name


def _edge_pairs(w, n, seed, tag):
    """Random w-bit pairs plus the operands that drive the longest carry and
    borrow chains: all ones, a lone top bit, zero, one."""
    top, ones = 1 << (w - 1), (1 << w) - 1
    ea = np.array([ones, ones, top, top, 0, ones, 1, top | 1], dtype=np.uint64)
    eb = np.array([ones, 1, top, ones, ones, 0, ones, ones], dtype=np.uint64)
    a, b = synth.int_pairs(n, w, seed, tag)
    return np.concatenate([ea, a]), np.concatenate([eb, b])


@pytest.mark.parametrize("w", [8, 9, 16, 17, 32])
def test_karatsuba_products(orc, toy, w):
    """Karatsuba (Algorithm "karatsuba" in the vector form of section V-B)
    against the integer product, at widths that recurse once (8, 9: odd
    split), twice (16, 17) and three times (32), with the edge operands
    that exercise the subtraction Z2 - (Z0 + Z1) over its full width; the
    oracle's gate counts equal the CUDA library's netlists."""
    from paper_2005_01945_gb300 import api, build
    build.build()
    p, P, kd, bk, ksk = toy
    a, b = _edge_pairs(w, 120 if w <= 9 else 24, 17, f"ka{w}")
    A = _enc_ints(orc, p, P, kd, a, w, f"kaa{w}")
    B = _enc_ints(orc, p, P, kd, b, w, f"kab{w}")
    want = [int(x) * int(y) for x, y in zip(a, b)]
    for name, kind in (("mul_karatsuba", api.MUL_KARATSUBA), ("mul_full", api.MUL_FULL)):
        R, g = getattr(orc, name)(P, bk, ksk, w, A, B)
        bits = orc.decrypt_bits(P, kd.s, R)
        got = [sum(int(v) << i for i, v in enumerate(row)) for row in bits]
        assert got == want, name
        assert g == len(a) * api.circuit_info(kind, w)[0], name
