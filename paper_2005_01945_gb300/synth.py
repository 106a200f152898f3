"""Seeded synthetic inputs for TFHE gate bootstrapping: raw random draws only.

This module holds none of the scheme's arithmetic.  It draws the random
numbers that key generation and encryption consume -- key bits, uniform
torus masks, discretised Gaussian noise -- and the plaintext bits and
integers of the workloads.  Both the GPU library's client helpers and the
CPU oracle take these arrays as inputs, so the two sides see identical draws
without sharing any code that computes on them.

Every stream is a numpy ``Generator(PCG64)`` seeded by a ``SeedSequence`` of
(master seed, purpose tag), so draws for one purpose never depend on how
many draws another purpose made.
"""
from __future__ import annotations

import zlib
from dataclasses import dataclass

import numpy as np

MASTER_SEED = 0x200501945


def _gen(seed: int, tag: str) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(
        np.random.SeedSequence([seed & 0xFFFFFFFFFFFF, zlib.crc32(tag.encode())])))


def uniform_torus32(g: np.random.Generator, shape) -> np.ndarray:
    """Uniform 32-bit words (uniform points of the discretised torus)."""
    return g.integers(0, 1 << 32, size=shape, dtype=np.uint64).astype(np.uint32)


def gaussian_torus32(g: np.random.Generator, shape, sigma: float) -> np.ndarray:
    """Centred Gaussian of standard deviation ``sigma`` (torus units),
    rounded to the nearest multiple of 2^-32, as int32 words."""
    if sigma == 0.0:
        return np.zeros(shape, dtype=np.int32)
    z = g.standard_normal(size=shape) * (sigma * 2.0 ** 32)
    return np.rint(z).astype(np.int64).astype(np.int32)


def key_bits(g: np.random.Generator, count: int) -> np.ndarray:
    return g.integers(0, 2, size=count, dtype=np.int32)


@dataclass
class TFHEParams:
    """Parameter set of the scheme (TFHE gate bootstrapping)."""
    n: int = 500            # LWE dimension
    N: int = 1024           # TLWE ring degree, k = 1
    l: int = 2              # gadget levels
    bg_bit: int = 10        # log2 Bg
    ks_t: int = 8           # key-switch levels
    ks_basebit: int = 2     # log2 key-switch base
    sigma_lwe: float = 2.0 ** -15
    sigma_bk: float = 2.0 ** -25

    @property
    def ks_digits(self) -> int:
        return (1 << self.ks_basebit) - 1


@dataclass
class KeyDraws:
    s: np.ndarray          # int32 [n]           LWE key bits
    S: np.ndarray          # int32 [N]           TLWE key bits
    bk_mask: np.ndarray    # uint32 [n][2l][N]   TLWE masks of every BK row
    bk_noise: np.ndarray   # int32  [n][2l][N]   TLWE noise of every BK row
    ksk_mask: np.ndarray   # uint32 [N][t][base-1][n]
    ksk_noise: np.ndarray  # int32  [N][t][base-1]


def key_draws(p: TFHEParams, seed: int = MASTER_SEED, *, noiseless: bool = False,
              zero_bk_mask: bool = False) -> KeyDraws:
    """Everything key generation draws.  ``noiseless`` zeroes both noise
    arrays; ``zero_bk_mask`` zeroes the BK masks (trivial TLWE rows)."""
    rows = 2 * p.l
    s = key_bits(_gen(seed, "lwe_key"), p.n)
    S = key_bits(_gen(seed, "tlwe_key"), p.N)
    bk_mask = uniform_torus32(_gen(seed, "bk_mask"), (p.n, rows, p.N))
    bk_noise = gaussian_torus32(_gen(seed, "bk_noise"), (p.n, rows, p.N),
                                0.0 if noiseless else p.sigma_bk)
    ksk_mask = uniform_torus32(_gen(seed, "ksk_mask"), (p.N, p.ks_t, p.ks_digits, p.n))
    ksk_noise = gaussian_torus32(_gen(seed, "ksk_noise"), (p.N, p.ks_t, p.ks_digits),
                                 0.0 if noiseless else p.sigma_lwe)
    if zero_bk_mask:
        bk_mask[:] = 0
    return KeyDraws(s, S, bk_mask, bk_noise, ksk_mask, ksk_noise)


@dataclass
class CtDraws:
    mask: np.ndarray   # uint32 [..., n]
    noise: np.ndarray  # int32  [...]


def ct_draws(p: TFHEParams, shape, seed: int, tag: str, *, noiseless: bool = False) -> CtDraws:
    """Masks and noise for encrypting ``shape`` bits under the LWE key."""
    shape = tuple(np.atleast_1d(np.asarray(shape, dtype=np.int64)).tolist())
    g = _gen(seed, "ct_" + tag)
    mask = uniform_torus32(g, shape + (p.n,))
    noise = gaussian_torus32(g, shape, 0.0 if noiseless else p.sigma_lwe)
    return CtDraws(mask, noise)


def random_bits(shape, seed: int, tag: str) -> np.ndarray:
    return _gen(seed, "bits_" + tag).integers(0, 2, size=shape, dtype=np.uint8)


def random_uints(shape, width: int, seed: int, tag: str) -> np.ndarray:
    """Uniform unsigned integers of ``width`` bits (uint64)."""
    return _gen(seed, "uint_" + tag).integers(0, 1 << width, size=shape, dtype=np.uint64)


def to_bits(x: np.ndarray, width: int) -> np.ndarray:
    """Integers -> bit planes, least significant first: shape x.shape + (width,)."""
    x = np.asarray(x, dtype=np.uint64)
    return ((x[..., None] >> np.arange(width, dtype=np.uint64)) & 1).astype(np.uint8)


def from_bits(b: np.ndarray) -> np.ndarray:
    """Inverse of ``to_bits`` along the last axis."""
    b = np.asarray(b, dtype=np.uint64)
    return (b << np.arange(b.shape[-1], dtype=np.uint64)).sum(axis=-1)


# Workload recipes (the input structure of each benchmark configuration).

GATES8_OPS = np.array([0, 0, 1, 1, 2, 2, 3, 3], dtype=np.uint8)  # NAND,NAND,AND,AND,OR,OR,XOR,XOR


def gates8_inputs(seed: int):
    """8 gates on 16 fresh encryptions of uniform bits: (ops, bits_a, bits_b)."""
    bits = random_bits((2, 8), seed, "gates8")
    return GATES8_OPS.copy(), bits[0], bits[1]


def int_pairs(batch: int, width: int, seed: int, tag: str):
    """``batch`` pairs of uniform ``width``-bit integers."""
    x = random_uints((2, batch), width, seed, tag)
    return x[0], x[1]
