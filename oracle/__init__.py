"""CPU oracle for TFHE gate bootstrapping (plain C, schoolbook products).

TEST INFRASTRUCTURE ONLY: importable from ``tests/``, from
``__graft_entry__.smoke()`` (as the checker) and from the cpu_baseline /
reference leg of ``bench.py``.  The product package never imports this
module and this module never imports the product package.

The arithmetic lives in ``tfhe_oracle.c`` (one translation unit, compiled
with gcc and OpenMP); this file only marshals numpy arrays.  Ciphertexts are
``uint32`` arrays of shape ``[..., n + 1]`` with the body ``b`` last.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tfhe_oracle.c")
_LIB = os.path.join(_HERE, "libtfhe_oracle.so")
_lock = threading.Lock()
_lib = None

NAND, AND, OR, XOR, NOR, XNOR, MAJ, ANDNY, ANDYN, ORNY, ORYN = range(11)
MU = 1 << 29  # 1/8 on the torus


class Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("N", ctypes.c_int32), ("l", ctypes.c_int32),
                ("bg_bit", ctypes.c_int32), ("ks_t", ctypes.c_int32),
                ("ks_basebit", ctypes.c_int32)]

    def astuple(self):
        return (self.n, self.N, self.l, self.bg_bit, self.ks_t, self.ks_basebit)


def default_params() -> Params:
    """LWE n=500; TLWE N=1024, k=1; Bg=2^10, l=2; key switch t=8, basebit=2."""
    return Params(500, 1024, 2, 10, 8, 2)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O3, OpenMP) if needed."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-Wall", "-Wextra", "-Wno-unused-parameter", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(Params)
        vp = ctypes.c_void_p
        i32, i64, u32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        sigs = {
            "orc_negacyclic_mul": (None, [i32, vp, vp, vp]),
            "orc_mul_by_xk": (None, [i32, vp, i32, vp]),
            "orc_modswitch": (i32, [i32, u32]),
            "orc_decompose_many": (None, [i32, i32, vp, i64, vp]),
            "orc_modswitch_many": (None, [i32, vp, i64, vp]),
            "orc_lwe_encrypt_bits": (None, [i32, vp, i64, vp, vp, vp, vp]),
            "orc_lwe_phase_many": (None, [i32, vp, i64, i64, vp, vp]),
            "orc_keygen_bk": (None, [P, vp, vp, vp, vp, vp]),
            "orc_keygen_ksk": (None, [P, vp, vp, vp, vp, vp]),
            "orc_gate_combine": (None, [i32, i32, vp, vp, vp]),
            "orc_gate_combine3": (None, [i32, i32, vp, vp, vp, vp]),
            "orc_gate3": (None, [P, vp, vp, i32, vp, vp, vp, vp]),
            "orc_add_maj": (i64, [P, vp, vp, i32, i64, vp, vp, vp, i32]),
            "orc_add_nw": (i64, [P, vp, vp, i32, i64, vp, vp, vp, i32]),
            "orc_mul_tree": (i64, [P, vp, vp, i32, i64, vp, vp, vp, i32]),
            "orc_mul_tree_maj": (i64, [P, vp, vp, i32, i64, vp, vp, vp, i32]),
            "orc_add_prefix": (i64, [P, vp, vp, i32, i64, vp, vp, vp, i32]),
            "orc_mul_dadda": (i64, [P, vp, vp, i32, i64, vp, vp, vp, i32]),
            "orc_mul_full": (i64, [P, vp, vp, i32, i64, vp, vp, vp, i32]),
            "orc_mul_karatsuba": (i64, [P, vp, vp, i32, i64, vp, vp, vp, i32]),
            "orc_blind_rotate_many": (None, [P, vp, i64, vp, u32, vp, i32]),
            "orc_sample_extract": (None, [i32, vp, vp]),
            "orc_keyswitch_many": (None, [P, vp, i64, vp, vp]),
            "orc_bootstrap_many": (None, [P, vp, vp, i64, vp, u32, vp, i32]),
            "orc_gates": (None, [P, vp, vp, i64, vp, vp, vp, vp, i32]),
            "orc_add": (i64, [P, vp, vp, i32, i64, vp, vp, vp, i32]),
            "orc_mul": (i64, [P, vp, vp, i32, i64, vp, vp, vp, i32]),
            "orc_matvec": (i64, [P, vp, vp, i32, i32, i32, vp, vp, vp, i32]),
            "orc_max_threads": (i32, []),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return ctypes.c_void_p(a.ctypes.data)


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a).astype(np.uint32, copy=False))


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a).astype(np.int32, copy=False))


# ---------------------------------------------------------------- primitives

def negacyclic_mul(a, b) -> np.ndarray:
    """a * b in Z[X]/(X^N+1) mod 2^32; a integer coefficients, b torus words."""
    a, b = _i32(a), _u32(b)
    out = np.empty_like(b)
    lib().orc_negacyclic_mul(len(b), _p(a), _p(b), _p(out))
    return out


def mul_by_xk(p, k: int) -> np.ndarray:
    p = _u32(p)
    out = np.empty_like(p)
    lib().orc_mul_by_xk(len(p), _p(p), int(k), _p(out))
    return out


def decompose(x, bg_bit: int, l: int) -> np.ndarray:
    x = _u32(x).ravel()
    d = np.empty((x.size, l), dtype=np.int32)
    lib().orc_decompose_many(bg_bit, l, _p(x), x.size, _p(d))
    return d


def modswitch(x, N: int) -> np.ndarray:
    x = _u32(x).ravel()
    out = np.empty(x.size, dtype=np.int32)
    lib().orc_modswitch_many(N, _p(x), x.size, _p(out))
    return out


# ---------------------------------------------------------------- client side

def encrypt_bits(P: Params, s, masks, noise, bits) -> np.ndarray:
    s, masks, noise = _i32(s), _u32(masks), _i32(noise)
    bits = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8))
    count = bits.size
    assert masks.shape[-1] == P.n and masks.size == count * P.n and noise.size == count
    out = np.empty(bits.shape + (P.n + 1,), dtype=np.uint32)
    lib().orc_lwe_encrypt_bits(P.n, _p(s), count, _p(masks), _p(noise), _p(bits), _p(out))
    return out


def phase(P: Params, s, cts) -> np.ndarray:
    """b - <a, s> of every ciphertext (last axis n+1 or wider, b at index n)."""
    s, cts = _i32(s), _u32(cts)
    stride = cts.shape[-1]
    count = cts.size // stride
    out = np.empty(cts.shape[:-1], dtype=np.uint32)
    lib().orc_lwe_phase_many(P.n, _p(s), count, stride, _p(cts), _p(out))
    return out


def decrypt_bits(P: Params, s, cts) -> np.ndarray:
    return (phase(P, s, cts).view(np.int32) > 0).astype(np.uint8)


def keygen_bk(P: Params, s, S, masks, noise) -> np.ndarray:
    rows = 2 * P.l
    s, S, masks, noise = _i32(s), _i32(S), _u32(masks), _i32(noise)
    assert masks.size == P.n * rows * P.N and noise.size == masks.size
    bk = np.empty((P.n, rows, 2, P.N), dtype=np.uint32)
    lib().orc_keygen_bk(ctypes.byref(P), _p(s), _p(S), _p(masks), _p(noise), _p(bk))
    return bk


def keygen_ksk(P: Params, s, S, masks, noise) -> np.ndarray:
    nd = (1 << P.ks_basebit) - 1
    s, S, masks, noise = _i32(s), _i32(S), _u32(masks), _i32(noise)
    assert masks.size == P.N * P.ks_t * nd * P.n and noise.size == P.N * P.ks_t * nd
    ksk = np.empty((P.N, P.ks_t, nd, P.n + 1), dtype=np.uint32)
    lib().orc_keygen_ksk(ctypes.byref(P), _p(s), _p(S), _p(masks), _p(noise), _p(ksk))
    return ksk


# ---------------------------------------------------------------- server side

def gate_combine(P: Params, op: int, ca, cb) -> np.ndarray:
    ca, cb = _u32(ca), _u32(cb)
    out = np.empty_like(ca)
    lib().orc_gate_combine(P.n, int(op), _p(ca), _p(cb), _p(out))
    return out


def blind_rotate(P: Params, bk, abar, mu: int = MU, nthreads: int = 0) -> np.ndarray:
    """abar: [count][n+1] mod-switched words -> acc [count][2][N]."""
    bk, abar = _u32(bk), _i32(abar)
    count = abar.size // (P.n + 1)
    acc = np.empty(abar.shape[:-1] + (2, P.N), dtype=np.uint32)
    lib().orc_blind_rotate_many(ctypes.byref(P), _p(bk), count, _p(abar), mu, _p(acc), nthreads)
    return acc


def sample_extract(P: Params, acc) -> np.ndarray:
    acc = _u32(acc)
    out = np.empty(P.N + 1, dtype=np.uint32)
    lib().orc_sample_extract(P.N, _p(acc), _p(out))
    return out


def keyswitch(P: Params, ksk, big) -> np.ndarray:
    """big: [count][N+1] LWE_N samples -> [count][n+1]."""
    ksk, big = _u32(ksk), _u32(big)
    count = big.size // (P.N + 1)
    out = np.empty(big.shape[:-1] + (P.n + 1,), dtype=np.uint32)
    lib().orc_keyswitch_many(ctypes.byref(P), _p(ksk), count, _p(big), _p(out))
    return out


def bootstrap(P: Params, bk, ksk, cts, mu: int = MU, nthreads: int = 0) -> np.ndarray:
    bk, ksk, cts = _u32(bk), _u32(ksk), _u32(cts)
    count = cts.size // (P.n + 1)
    out = np.empty_like(cts)
    lib().orc_bootstrap_many(ctypes.byref(P), _p(bk), _p(ksk), count, _p(cts), mu, _p(out),
                             nthreads)
    return out


def gates(P: Params, bk, ksk, ops, ca, cb, nthreads: int = 0) -> np.ndarray:
    bk, ksk, ca, cb = _u32(bk), _u32(ksk), _u32(ca), _u32(cb)
    ops = np.ascontiguousarray(np.asarray(ops, dtype=np.uint8))
    count = ops.size
    assert ca.size == count * (P.n + 1) and cb.size == ca.size
    out = np.empty_like(ca)
    lib().orc_gates(ctypes.byref(P), _p(bk), _p(ksk), count, _p(ops), _p(ca), _p(cb), _p(out),
                    nthreads)
    return out


def add(P: Params, bk, ksk, w: int, A, B, nthreads: int = 0):
    """A, B: [batch][w][n+1] -> (R, gates)."""
    bk, ksk, A, B = _u32(bk), _u32(ksk), _u32(A), _u32(B)
    batch = A.size // (w * (P.n + 1))
    R = np.empty_like(A)
    g = lib().orc_add(ctypes.byref(P), _p(bk), _p(ksk), w, batch, _p(A), _p(B), _p(R), nthreads)
    return R, int(g)


def _circuit(name, P, bk, ksk, w, A, B, nthreads):
    bk, ksk, A, B = _u32(bk), _u32(ksk), _u32(A), _u32(B)
    batch = A.size // (w * (P.n + 1))
    R = np.empty_like(A)
    g = getattr(lib(), name)(ctypes.byref(P), _p(bk), _p(ksk), w, batch, _p(A), _p(B), _p(R),
                             nthreads)
    return R, int(g)


def add_maj(P: Params, bk, ksk, w: int, A, B, nthreads: int = 0):
    """Ripple adder with majority-gate carries -> (R, gates)."""
    return _circuit("orc_add_maj", P, bk, ksk, w, A, B, nthreads)


def add_nw(P: Params, bk, ksk, w: int, A, B, nthreads: int = 0):
    """The paper's number-wise adder GPU_n -> (R, gates)."""
    return _circuit("orc_add_nw", P, bk, ksk, w, A, B, nthreads)


def mul_tree(P: Params, bk, ksk, w: int, A, B, nthreads: int = 0):
    """Multiplication with tree-based accumulation -> (R, gates)."""
    return _circuit("orc_mul_tree", P, bk, ksk, w, A, B, nthreads)


def mul_tree_maj(P: Params, bk, ksk, w: int, A, B, nthreads: int = 0):
    """Tree-accumulated multiplication with majority-carry adders -> (R, gates)."""
    return _circuit("orc_mul_tree_maj", P, bk, ksk, w, A, B, nthreads)


def add_prefix(P: Params, bk, ksk, w: int, A, B, nthreads: int = 0):
    """Sklansky parallel-prefix adder (majority gates) -> (R, gates)."""
    return _circuit("orc_add_prefix", P, bk, ksk, w, A, B, nthreads)


def mul_dadda(P: Params, bk, ksk, w: int, A, B, nthreads: int = 0):
    """Truncated multiplication by a Dadda tree and a prefix adder -> (R, gates)."""
    return _circuit("orc_mul_dadda", P, bk, ksk, w, A, B, nthreads)


def _full(name, P, bk, ksk, w, A, B, nthreads):
    bk, ksk, A, B = _u32(bk), _u32(ksk), _u32(A), _u32(B)
    batch = A.size // (w * (P.n + 1))
    R = np.empty((batch, 2 * w, P.n + 1), dtype=np.uint32)
    g = getattr(lib(), name)(ctypes.byref(P), _p(bk), _p(ksk), w, batch, _p(A), _p(B), _p(R),
                             nthreads)
    return R, int(g)


def mul_full(P: Params, bk, ksk, w: int, A, B, nthreads: int = 0):
    """Full product (2w bits), partial products summed by the tree ->
    (R [batch][2w][n+1], gates)."""
    return _full("orc_mul_full", P, bk, ksk, w, A, B, nthreads)


def mul_karatsuba(P: Params, bk, ksk, w: int, A, B, nthreads: int = 0):
    """Karatsuba full product (2w bits) -> (R [batch][2w][n+1], gates)."""
    return _full("orc_mul_karatsuba", P, bk, ksk, w, A, B, nthreads)


def gate3(P: Params, bk, ksk, op: int, ca, cb, cc) -> np.ndarray:
    """One 3-input gate per row: ca, cb, cc are [n+1] or [count][n+1]."""
    ca, cb, cc, bk, ksk = _u32(ca), _u32(cb), _u32(cc), _u32(bk), _u32(ksk)
    if not (ca.shape == cb.shape == cc.shape and ca.shape[-1] == P.n + 1 and ca.ndim <= 2):
        raise ValueError("gate3: ca, cb, cc must be matching [n+1] or [count][n+1] arrays")
    out = np.empty_like(ca)
    rows = (ca, cb, cc, out) if ca.ndim == 1 else None
    for a, b, c, o in ([rows] if rows else zip(ca, cb, cc, out)):
        lib().orc_gate3(ctypes.byref(P), _p(bk), _p(ksk), int(op), _p(a), _p(b), _p(c), _p(o))
    return out


def gate_combine3(P: Params, op: int, ca, cb, cc) -> np.ndarray:
    ca, cb, cc = _u32(ca), _u32(cb), _u32(cc)
    out = np.empty_like(ca)
    lib().orc_gate_combine3(P.n, int(op), _p(ca), _p(cb), _p(cc), _p(out))
    return out


def mul(P: Params, bk, ksk, w: int, A, B, nthreads: int = 0):
    bk, ksk, A, B = _u32(bk), _u32(ksk), _u32(A), _u32(B)
    batch = A.size // (w * (P.n + 1))
    R = np.empty_like(A)
    g = lib().orc_mul(ctypes.byref(P), _p(bk), _p(ksk), w, batch, _p(A), _p(B), _p(R), nthreads)
    return R, int(g)


def matvec(P: Params, bk, ksk, w: int, M, v, nthreads: int = 0):
    """M: [rows][cols][w][n+1], v: [cols][w][n+1] -> (Y [rows][w][n+1], gates)."""
    bk, ksk, M, v = _u32(bk), _u32(ksk), _u32(M), _u32(v)
    rows, cols = M.shape[0], M.shape[1]
    Y = np.empty((rows, w, P.n + 1), dtype=np.uint32)
    g = lib().orc_matvec(ctypes.byref(P), _p(bk), _p(ksk), w, rows, cols, _p(M), _p(v), _p(Y),
                         nthreads)
    return Y, int(g)


def max_threads() -> int:
    return int(lib().orc_max_threads())
