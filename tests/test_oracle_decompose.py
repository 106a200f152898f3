"""Pins for rounding: the signed gadget decomposition and the mod switch.

The decomposition is checked by its defining properties (digit range and
reconstruction within half a step) and, on a toy word layout, against a
brute-force search over every digit tuple.  The mod switch is checked
against a brute-force nearest-point search on the 2N-gon.
"""
import itertools

import numpy as np
import pytest

M32 = 1 << 32


def _edge_values(step):
    vals = [0, 1, M32 - 1, 1 << 31, (1 << 31) - 1, step, step - 1, step // 2, step // 2 - 1,
            step // 2 + 1, M32 - step // 2, M32 - step // 2 - 1]
    return [v % M32 for v in vals]


@pytest.mark.parametrize("bg_bit,l", [(10, 2), (8, 3), (4, 4), (2, 1)])
def test_decomposition_reconstruction(orc, bg_bit, l):
    rng = np.random.default_rng(bg_bit * 10 + l)
    step = 1 << (32 - bg_bit * l)
    x = np.concatenate([rng.integers(0, M32, size=100_000, dtype=np.uint64),
                        np.array(_edge_values(step), dtype=np.uint64)]).astype(np.uint32)
    d = orc.decompose(x, bg_bit, l).astype(np.int64)
    half = 1 << (bg_bit - 1)
    assert d.min() >= -half and d.max() < half
    weights = np.array([1 << (32 - bg_bit * (j + 1)) for j in range(l)], dtype=np.int64)
    recon = (d * weights).sum(axis=1)
    err = (recon - x.astype(np.int64)) % M32
    err = np.where(err >= M32 // 2, err - M32, err)
    assert np.abs(err).max() <= step // 2
    # ties round up: x exactly half a step above a multiple reconstructs above x
    tie = np.array([(step // 2 + k * step) % M32 for k in range(0, 50)], dtype=np.uint32)
    dt = orc.decompose(tie, bg_bit, l).astype(np.int64)
    et = ((dt * weights).sum(axis=1) - tie.astype(np.int64)) % M32
    assert np.all(et == step // 2)


def test_decomposition_brute_force_toy():
    """bg_bit = 2, l = 3 (precision 6 bits): for x = m * 2^24 + r the digits
    must be the unique tuple in [-2, 1]^3 whose value is nearest to x."""
    import oracle
    bg_bit, l = 2, 3
    step = 1 << (32 - bg_bit * l)
    tuples = list(itertools.product(range(-2, 2), repeat=l))
    xs = []
    for m in range(64):
        for r in (0, 1, step // 2 - 1, step // 2, step // 2 + 1, step - 1):
            xs.append((m * step + r) % M32)
    got = oracle.decompose(np.array(xs, dtype=np.uint32), bg_bit, l)
    for x, dg in zip(xs, got):
        best = None
        for t in tuples:
            v = sum(t[j] << (32 - bg_bit * (j + 1)) for j in range(l)) % M32
            dist = (v - x) % M32
            dist = dist - M32 if dist >= M32 // 2 else dist  # signed distance v - x
            key = (abs(dist), -dist)                           # ties: prefer v above x
            if best is None or key < best[0]:
                best = (key, t)
        assert tuple(int(v) for v in dg) == best[1], (x, dg, best)


@pytest.mark.parametrize("N", [16, 1024])
def test_modswitch_nearest_point(orc, N):
    rng = np.random.default_rng(N)
    step = M32 // (2 * N)
    xs = np.concatenate([rng.integers(0, M32, size=2000 if N <= 64 else 200, dtype=np.uint64),
                         np.array(_edge_values(step), dtype=np.uint64)]).astype(np.uint32)
    got = orc.modswitch(xs, N)
    for x, g in zip(xs.tolist(), got.tolist()):
        # nearest k/2N to x/2^32 on the circle, ties towards the larger k
        best = min(range(2 * N), key=lambda k: (abs(((k * step - x + M32 // 2) % M32) - M32 // 2),
                                                 -(((k * step - x + M32 // 2) % M32) - M32 // 2)))
        assert g == best, (x, g, best)
