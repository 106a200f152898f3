"""Pins for the oracle's polynomial arithmetic in Z[X]/(X^N+1) mod 2^32.

Each check uses an independent computation: Karatsuba multiplication on
Python integers followed by the X^N = -1 fold, numpy's convolution, and the
closed form of monomial products.
"""
import numpy as np
import pytest

M32 = 1 << 32


def karatsuba(x, y):
    """Full product of two coefficient lists (equal power-of-two length)."""
    n = len(x)
    if n <= 2:
        out = [0] * (2 * n - 1)
        for i in range(n):
            for j in range(n):
                out[i + j] += x[i] * y[j]
        return out
    h = n // 2
    x0, x1, y0, y1 = x[:h], x[h:], y[:h], y[h:]
    z0 = karatsuba(x0, y0)
    z2 = karatsuba(x1, y1)
    z1 = karatsuba([a + b for a, b in zip(x0, x1)], [a + b for a, b in zip(y0, y1)])
    mid = [a - b - c for a, b, c in zip(z1, z0, z2)]
    out = [0] * (2 * n - 1)
    for i, v in enumerate(z0):
        out[i] += v
    for i, v in enumerate(mid):
        out[i + h] += v
    for i, v in enumerate(z2):
        out[i + 2 * h] += v
    return out


def fold_negacyclic(full, N):
    return [(full[k] - (full[k + N] if k + N < len(full) else 0)) % M32 for k in range(N)]


@pytest.mark.parametrize("N", [4, 8, 16, 32, 64])
def test_negacyclic_vs_karatsuba(orc, N):
    rng = np.random.default_rng(N)
    for trial in range(20):
        a = rng.integers(-512, 512, size=N).astype(np.int32)
        b = rng.integers(0, M32, size=N, dtype=np.uint64).astype(np.uint32)
        ref = fold_negacyclic(karatsuba([int(v) for v in a], [int(v) for v in b]), N)
        got = orc.negacyclic_mul(a, b)
        assert got.tolist() == ref


def test_negacyclic_vs_numpy_convolution_full_size(orc):
    """N = 1024 with 10-bit signed digits times 32-bit words: split the words
    into 16-bit halves so every convolution is exact in int64."""
    N = 1024
    rng = np.random.default_rng(7)
    a = rng.integers(-512, 512, size=N).astype(np.int64)
    b = rng.integers(0, M32, size=N, dtype=np.uint64)
    lo, hi = (b & 0xFFFF).astype(np.int64), (b >> 16).astype(np.int64)
    full_lo, full_hi = np.convolve(a, lo), np.convolve(a, hi)
    full = [int(x) + (int(y) << 16) for x, y in zip(full_lo, full_hi)]
    ref = fold_negacyclic(full, N)
    got = orc.negacyclic_mul(a.astype(np.int32), b.astype(np.uint32))
    assert got.tolist() == ref


@pytest.mark.parametrize("N", [8, 32])
def test_monomial_products(orc, N):
    """X^i * X^j = X^(i+j) for i+j < N and -X^(i+j-N) otherwise."""
    for i in range(N):
        for j in range(N):
            a = np.zeros(N, np.int32)
            b = np.zeros(N, np.uint32)
            a[i] = 1
            b[j] = 1
            got = orc.negacyclic_mul(a, b)
            want = np.zeros(N, np.uint32)
            if i + j < N:
                want[i + j] = 1
            else:
                want[i + j - N] = M32 - 1
            assert np.array_equal(got, want), (i, j)


def test_identity_and_distributivity(orc):
    N = 64
    rng = np.random.default_rng(3)
    b = rng.integers(0, M32, size=N, dtype=np.uint64).astype(np.uint32)
    one = np.zeros(N, np.int32)
    one[0] = 1
    assert np.array_equal(orc.negacyclic_mul(one, b), b)
    a1 = rng.integers(-1000, 1000, size=N).astype(np.int32)
    a2 = rng.integers(-1000, 1000, size=N).astype(np.int32)
    lhs = orc.negacyclic_mul((a1 + a2).astype(np.int32), b)
    rhs = orc.negacyclic_mul(a1, b) + orc.negacyclic_mul(a2, b)  # uint32 wrap
    assert np.array_equal(lhs, rhs)


@pytest.mark.parametrize("N", [16, 1024])
def test_mul_by_xk_closed_form(orc, N):
    """X^k p: for k < N the coefficients shift up by k and the k that wrap
    past X^N come back negated at the bottom; X^(k+N) p = -X^k p."""
    rng = np.random.default_rng(N)
    p = rng.integers(0, M32, size=N, dtype=np.uint64).astype(np.uint32)
    ks = range(2 * N) if N <= 64 else [0, 1, 5, N - 1, N, N + 3, 2 * N - 1]
    for k in ks:
        kk = k % N
        shifted = np.concatenate([(np.uint32(0) - p[N - kk:]).astype(np.uint32), p[:N - kk]])
        if k >= N:
            shifted = (np.uint32(0) - shifted).astype(np.uint32)
        assert np.array_equal(orc.mul_by_xk(p, k), shifted), k
    # X^(2N) = 1 and X^N = -1 as polynomial products too
    assert np.array_equal(orc.mul_by_xk(p, 2 * N), p)
    e = np.zeros(N, np.int32)
    if N <= 64:
        for k in range(N):
            e[:] = 0
            e[k] = 1
            assert np.array_equal(orc.mul_by_xk(p, k), orc.negacyclic_mul(e, p))
