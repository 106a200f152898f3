import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


def toy_params(n=8, N=32):
    """Small parameter set for brute-force pins (same gadget/KS shape)."""
    from paper_2005_01945_gb300.synth import TFHEParams
    return TFHEParams(n=n, N=N)


def oparams(p):
    import oracle
    return oracle.Params(p.n, p.N, p.l, p.bg_bit, p.ks_t, p.ks_basebit)


@pytest.fixture(scope="session")
def full_keys(orc):
    """Oracle keys for the default parameter set, from the master seed."""
    from paper_2005_01945_gb300 import synth
    p = synth.TFHEParams()
    kd = synth.key_draws(p, synth.MASTER_SEED)
    P = oparams(p)
    bk = orc.keygen_bk(P, kd.s, kd.S, kd.bk_mask, kd.bk_noise)
    ksk = orc.keygen_ksk(P, kd.s, kd.S, kd.ksk_mask, kd.ksk_noise)
    return p, P, kd, bk, ksk


def center(x):
    """uint32 torus words -> signed int64 representative in [-2^31, 2^31)."""
    return np.asarray(x, dtype=np.uint32).view(np.int32).astype(np.int64)


def np_negacyclic(a, b):
    """Independent negacyclic product mod 2^32 via numpy convolutions:
    a small signed integers, b uint32 words split into 16-bit halves so each
    convolution is exact in int64."""
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.uint32).astype(np.uint64)
    N = len(b)
    out = np.zeros(N, dtype=object)
    for shift, half in ((0, (b & 0xFFFF).astype(np.int64)), (16, (b >> 16).astype(np.int64))):
        full = np.convolve(a, half).astype(object) * (1 << shift)
        out[:N] += full[:N]
        out[:N - 1] -= full[N:]
    return np.array([int(v) % (1 << 32) for v in out], dtype=np.uint32)


def trivial_rotation(mu, N, m):
    """X^m * (mu + mu X + ... + mu X^(N-1)) for m in [0, 2N), as uint32."""
    m %= 2 * N
    k = np.arange(N)
    sign = np.where(k >= (m % N), 1, -1)
    if m >= N:
        sign = -sign
    return (sign * mu).astype(np.int64).astype(np.uint32)
