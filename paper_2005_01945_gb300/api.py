"""Thin Python binding of libtfhe_gb.so (ctypes; argument marshalling only).

Every computation runs in the library's CUDA kernels.  Device arrays are
torch CUDA tensors (PyTorch provides device memory and streams); host
arrays for key upload may be numpy arrays.  If the library has not been
built this module raises on first use -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .synth import TFHEParams

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtfhe_gb.so")

LWE_STRIDE = 512
BIG_STRIDE = 1056
MU = 1 << 29
NOALLOC_MAX_GATES = 512
NAND, AND, OR, XOR, NOR, XNOR, MAJ, ANDNY, ANDYN, ORNY, ORYN = range(11)
GATE_NAMES = ["NAND", "AND", "OR", "XOR", "NOR", "XNOR", "MAJ", "ANDNY", "ANDYN", "ORNY", "ORYN"]

_STATUS = {0: "TFHE_OK", -1: "TFHE_EINVAL", -2: "TFHE_ENOMEM", -3: "TFHE_ECUDA",
           -4: "TFHE_ETIMEOUT", -5: "TFHE_EBUSY", -6: "TFHE_EDEVICE", -7: "TFHE_ECANCELED"}


class TFHEError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class CParams(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in ("n", "N", "k", "l", "bg_bit", "ks_t", "ks_basebit")]

    @classmethod
    def of(cls, p: TFHEParams) -> "CParams":
        return cls(p.n, p.N, 1, p.l, p.bg_bit, p.ks_t, p.ks_basebit)


EXPORTS = {
    # name: (restype, argtypes)
    "tfhe_ctx_create": (ctypes.c_int, [ctypes.POINTER(CParams), ctypes.c_int, ctypes.c_void_p]),
    "tfhe_ctx_set_keys": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "tfhe_ctx_destroy": (None, [ctypes.c_void_p]),
    "tfhe_ctx_save_keys": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "tfhe_ctx_load_keys": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "tfhe_last_error": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]),
    "tfhe_ctx_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32)]),
    "tfhe_bootstrap_gates": (ctypes.c_int, [ctypes.c_void_p] * 5 + [ctypes.c_size_t, ctypes.c_void_p]),
    "tfhe_bootstrap_gates_noalloc": (ctypes.c_int, [ctypes.c_void_p] * 5 + [ctypes.c_size_t,
                                                                           ctypes.c_void_p]),
    "tfhe_bootstrap": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_size_t, ctypes.c_uint32,
                                                             ctypes.c_void_p]),
    "tfhe_blind_rotate_extract": (ctypes.c_int, [ctypes.c_void_p] * 5 + [ctypes.c_size_t,
                                                                        ctypes.c_void_p]),
    "tfhe_keyswitch": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_size_t, ctypes.c_void_p]),
    "tfhe_tc_key_bytes": (ctypes.c_size_t, []),
    "tfhe_tc_digit_bytes": (ctypes.c_size_t, [ctypes.c_size_t]),
    "tfhe_tc_prepare_key": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "tfhe_cmux_products_tc": (ctypes.c_int, [ctypes.c_void_p] * 5 + [ctypes.c_size_t,
                                                                     ctypes.c_void_p]),
    "tfhe_add_n": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 3
                   + [ctypes.c_size_t, ctypes.c_void_p]),
    "tfhe_mul_n": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 3
                   + [ctypes.c_size_t, ctypes.c_void_p]),
    "tfhe_matvec": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
                    + [ctypes.c_void_p] * 4),
    "tfhe_run_jobs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                     ctypes.c_void_p]),
    "tfhe_schedule_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                          ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int64)]),
    "tfhe_circuit_info": (ctypes.c_int, [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_int64),
                                                               ctypes.POINTER(ctypes.c_int32)]),
    "tfhe_circuit_eval_plain": (ctypes.c_int, [ctypes.c_int] * 4 + [ctypes.c_void_p,
                                                                     ctypes.c_size_t,
                                                                     ctypes.c_void_p,
                                                                     ctypes.c_size_t]),
    "tfhe_ctx_set_option": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64]),
    "tfhe_ctx_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_void_p]),
    "tfhe_ctx_launches": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "tfhe_ctx_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int64)]),
    "tfhe_serve_start": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t]),
    "tfhe_serve_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_uint64)]),
    "tfhe_serve_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64,
                                       ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_double)]),
    "tfhe_serve_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double)]),
    "tfhe_serve_cancel": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "tfhe_serve_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "tfhe_serve_latencies": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                            ctypes.POINTER(ctypes.c_size_t)]),
    "tfhe_serve_select": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_size_t, ctypes.c_int64,
                                                               ctypes.c_int32, ctypes.c_void_p,
                                                               ctypes.c_float, ctypes.c_void_p,
                                                               ctypes.POINTER(ctypes.c_size_t)]),
    "tfhe_serve_stop": (ctypes.c_int, [ctypes.c_void_p]),
    "tfhe_keygen": (ctypes.c_int, [ctypes.POINTER(CParams)] + [ctypes.c_void_p] * 9),
    "tfhe_encrypt_bits": (ctypes.c_int, [ctypes.POINTER(CParams)] + [ctypes.c_void_p] * 5
                          + [ctypes.c_size_t, ctypes.c_void_p]),
    "tfhe_phase": (ctypes.c_int, [ctypes.POINTER(CParams)] + [ctypes.c_void_p] * 3
                   + [ctypes.c_size_t, ctypes.c_void_p]),
}

GATE, ADD, MUL, MATVEC, ADD_MAJ, ADD_NW, MUL_TREE, MUL_FULL, MUL_KARATSUBA, MUL_TREE_MAJ, \
    ADD_PREFIX, MUL_DADDA = range(12)
OPT_GRAPHS, OPT_PER_GATE, OPT_PROFILE, OPT_BR_GROUP, OPT_SCHEDULE, OPT_LEVEL_WIDTH, \
    OPT_KS_KERNEL, OPT_TEST_KS_STALL, OPT_TEST_FREE_HBM = range(9)
KS_TILED = 64   # OPT_KS_KERNEL value of the tiled key-switch kernel
SCHED_ASAP, SCHED_BALANCED = 0, 1


class CJob(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("width", ctypes.c_int32), ("rows", ctypes.c_int32),
                ("cols", ctypes.c_int32), ("batch", ctypes.c_int64), ("in0", ctypes.c_void_p),
                ("in1", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class CRequest(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("width", ctypes.c_int32), ("rows", ctypes.c_int32),
                ("cols", ctypes.c_int32), ("in0", ctypes.c_void_p), ("in1", ctypes.c_void_p),
                ("out", ctypes.c_void_p)]


class CServeInfo(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in ("submitted", "completed", "failed", "gates",
                                               "iterations", "in_flight", "queued")] + \
               [("wall_ms", ctypes.c_double)] + \
               [(f, ctypes.c_uint64) for f in ("pool_bytes", "pool_cap_bytes", "pool_grows",
                                               "admitted_busy", "cancelled")]


_lib = None


def lib():
    """Load libtfhe_gb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to the library must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    if not x.is_contiguous():
        raise ValueError("tensors passed to the library must be contiguous")
    return ctypes.c_void_p(x.data_ptr())


def _dev(x, dtype=None):
    """Device pointer of a contiguous CUDA tensor; anything else is refused
    (the library computes on the GPU only)."""
    import torch
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"expected a CUDA tensor, got {type(x).__name__}"
                        + (f" on {x.device}" if isinstance(x, torch.Tensor) else ""))
    if dtype is not None and x.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {x.dtype}")
    if not x.is_contiguous():
        raise ValueError("tensors passed to the library must be contiguous")
    return ctypes.c_void_p(x.data_ptr())


def _need(x, rows, name, stride=LWE_STRIDE):
    """Refuse a buffer that holds fewer than rows x stride words: the library
    trusts the sizes it is given, so a short buffer would be overrun on the
    device."""
    if x is not None and x.numel() < rows * stride:
        raise TFHEError(-1, f"{name} holds {x.numel()} words, needs {rows} x {stride}")


def job_rows(kind, width, rows=0, cols=0):
    """Ciphertext rows (in0, in1, out) of one instance of a circuit job:
    GATE 1, 1, 1; MATVEC rows*cols*w, cols*w, rows*w; full products w, w,
    2w; every other circuit w, w, w."""
    if kind == GATE:
        return 1, 1, 1
    if kind == MATVEC:
        return rows * cols * width, cols * width, rows * width
    if kind in (MUL_FULL, MUL_KARATSUBA):
        return width, width, 2 * width
    return width, width, width


def _need_job(batch, kind, width, rows, cols, in0, in1, out):
    r0, r1, ro = job_rows(kind, width, rows, cols)
    if batch > 0 and min(r0, r1, ro) > 0:
        _need(in0, batch * r0, "in0")
        _need(in1, batch * r1, "in1")
        _need(out, batch * ro, "out")


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(rc, ctx=None):
    if rc != 0:
        msg = ""
        if ctx is not None:
            buf = ctypes.create_string_buffer(512)
            lib().tfhe_last_error(ctx, buf, 512)
            msg = buf.value.decode(errors="replace")
        raise TFHEError(rc, msg)


class Context:
    """A device context holding the bootstrapping and key-switching keys."""

    def __init__(self, params: TFHEParams | None = None, device: int = 0):
        self.params = params or TFHEParams()
        self.cparams = CParams.of(self.params)
        self.device = device
        h = ctypes.c_void_p()
        _check(lib().tfhe_ctx_create(ctypes.byref(self.cparams), device, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().tfhe_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, rc):
        _check(rc, self._h)

    def set_keys(self, bk, ksk, stream=None):
        """bk int32 [n][4][2][N], ksk int32 [N][t][3][n+1]; host or device."""
        self._c(lib().tfhe_ctx_set_keys(self._h, _ptr(bk), _ptr(ksk), _stream(stream)))

    def save_keys(self, path):
        """Write the device keys (NTT-domain bootstrapping key, padded
        key-switching key) with a checked header to `path`."""
        self._c(lib().tfhe_ctx_save_keys(self._h, os.fsencode(path)))

    def load_keys(self, path):
        """Load keys written by save_keys for the same parameters."""
        self._c(lib().tfhe_ctx_load_keys(self._h, os.fsencode(path)))

    def status(self) -> int:
        code = ctypes.c_uint32(0)
        rc = lib().tfhe_ctx_status(self._h, ctypes.byref(code))
        if rc not in (0, -6):
            self._c(rc)
        return int(code.value)

    def bootstrap_gates(self, ops, a, b, out, stream=None):
        import torch
        count = ops.numel()
        for t, name in ((a, "a"), (b, "b"), (out, "out")):
            _need(t, count, name)
        self._c(lib().tfhe_bootstrap_gates(self._h, _dev(ops, torch.uint8), _dev(a, torch.int32),
                                           _dev(b, torch.int32), _dev(out, torch.int32), count,
                                           _stream(stream)))

    def bootstrap_gates_noalloc(self, ops, a, b, out, stream=None):
        """Like bootstrap_gates, but the library allocates nothing during the
        call (fixed scratch of NOALLOC_MAX_GATES gates per device; calls that
        overlap on the GPU race)."""
        import torch
        count = ops.numel()
        for t, name in ((a, "a"), (b, "b"), (out, "out")):
            _need(t, count, name)
        self._c(lib().tfhe_bootstrap_gates_noalloc(
            self._h, _dev(ops, torch.uint8), _dev(a, torch.int32), _dev(b, torch.int32),
            _dev(out, torch.int32), count, _stream(stream)))

    def bootstrap(self, x, out, mu=MU, stream=None):
        import torch
        count = x.shape[0]
        _need(x, count, "x")
        _need(out, count, "out")
        self._c(lib().tfhe_bootstrap(self._h, _dev(x, torch.int32), _dev(out, torch.int32), count,
                                     mu, _stream(stream)))

    def blind_rotate_extract(self, ops, a, b, big, stream=None):
        import torch
        count = a.shape[0]
        _need(a, count, "a")
        _need(b, count, "b")
        _need(ops, count, "ops", 1)
        _need(big, count, "big", BIG_STRIDE)
        self._c(lib().tfhe_blind_rotate_extract(
            self._h, None if ops is None else _dev(ops, torch.uint8), _dev(a, torch.int32),
            None if b is None else _dev(b, torch.int32), _dev(big, torch.int32), count,
            _stream(stream)))

    def keyswitch(self, big, out, stream=None):
        import torch
        _need(big, big.shape[0], "big", BIG_STRIDE)
        _need(out, big.shape[0], "out")
        self._c(lib().tfhe_keyswitch(self._h, _dev(big, torch.int32), _dev(out, torch.int32),
                                     big.shape[0], _stream(stream)))

    def tc_prepare_key(self, bk_rows, key_ops, stream=None):
        """bk_rows: uint32 (as int32) [4][2][1024] device tensor -> key_ops
        (uint8 device tensor of tc_key_bytes() bytes)."""
        import torch
        if bk_rows.numel() < 4 * 2 * 1024 or key_ops.numel() * key_ops.element_size() < \
                lib().tfhe_tc_key_bytes():
            raise TFHEError(-1, "tc_prepare_key: buffer too small")
        self._c(lib().tfhe_tc_prepare_key(self._h, _dev(bk_rows, torch.int32), _dev(key_ops),
                                          _stream(stream)))

    def cmux_products_tc(self, digits, key_ops, digit_ops, out, stream=None):
        """digits: int32 [count][4][1024]; out: int32 (uint32 words)
        [count][2][1024]; count a multiple of 128."""
        import torch
        count = digits.shape[0]
        if digits.numel() < count * 4096 or out.numel() < count * 2048 or \
                digit_ops.numel() * digit_ops.element_size() < lib().tfhe_tc_digit_bytes(count):
            raise TFHEError(-1, "cmux_products_tc: buffer too small")
        self._c(lib().tfhe_cmux_products_tc(self._h, _dev(digits, torch.int32), _dev(key_ops),
                                            _dev(digit_ops), _dev(out, torch.int32), count,
                                            _stream(stream)))

    def add_n(self, width, A, B, R, stream=None):
        import torch
        batch = A.shape[0]
        _need_job(batch, ADD, width, 0, 0, A, B, R)
        self._c(lib().tfhe_add_n(self._h, width, _dev(A, torch.int32), _dev(B, torch.int32),
                                 _dev(R, torch.int32), batch, _stream(stream)))

    def mul_n(self, width, A, B, R, stream=None):
        import torch
        batch = A.shape[0]
        _need_job(batch, MUL, width, 0, 0, A, B, R)
        self._c(lib().tfhe_mul_n(self._h, width, _dev(A, torch.int32), _dev(B, torch.int32),
                                 _dev(R, torch.int32), batch, _stream(stream)))

    def matvec(self, width, M, v, y, stream=None):
        import torch
        rows, cols = M.shape[0], M.shape[1]
        _need_job(1, MATVEC, width, rows, cols, M, v, y)
        self._c(lib().tfhe_matvec(self._h, width, rows, cols, _dev(M, torch.int32),
                                  _dev(v, torch.int32), _dev(y, torch.int32), _stream(stream)))


    def run_jobs(self, jobs, stream=None):
        """jobs: list of dicts kind, width, [rows, cols], batch, in0, in1, out
        (device tensors).  All jobs share one level schedule."""
        arr = (CJob * len(jobs))()
        for k, j in enumerate(jobs):
            _need_job(j["batch"], j["kind"], j["width"], j.get("rows", 0), j.get("cols", 0),
                      j["in0"], j["in1"], j["out"])
            arr[k] = CJob(j["kind"], j["width"], j.get("rows", 0), j.get("cols", 0), j["batch"],
                          _dev(j["in0"]).value, _dev(j["in1"]).value, _dev(j["out"]).value)
        self._c(lib().tfhe_run_jobs(self._h, arr, len(jobs), _stream(stream)))

    def set_option(self, option, value):
        self._c(lib().tfhe_ctx_set_option(self._h, option, int(value)))

    def autotune(self, cache_path=None) -> dict:
        """Pick blind-rotation group sizes and key-switch j-splits per level
        width by timing them on this device (results are unchanged)."""
        ch = np.zeros(16, dtype=np.int32)
        self._c(lib().tfhe_ctx_autotune(self._h, cache_path.encode() if cache_path else None,
                                        ctypes.c_void_p(ch.ctypes.data)))
        edges = ["<=152", "<=304", "<=608", "<=1216", "<=2432", "<=4864", "<=9728", ">9728"]
        return {"br_group": dict(zip(edges, ch[:8].tolist())),
                "ks_chunks": dict(zip(edges, ch[8:].tolist()))}

    def launches(self) -> int:
        v = ctypes.c_uint64(0)
        self._c(lib().tfhe_ctx_launches(self._h, ctypes.byref(v)))
        return int(v.value)

    def profile(self) -> dict:
        """Device time of blind-rotation / key-switch launches of the last
        schedule runs (TFHE_OPT_PROFILE must be on); resets."""
        bt, kt = ctypes.c_double(0), ctypes.c_double(0)
        bl, bb, kl = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
        self._c(lib().tfhe_ctx_profile(self._h, ctypes.byref(bt), ctypes.byref(bl),
                                       ctypes.byref(bb), ctypes.byref(kt), ctypes.byref(kl)))
        return dict(br_ms=bt.value, br_launches=bl.value, br_bootstraps=bb.value,
                    ks_ms=kt.value, ks_launches=kl.value)


    # ---- serving (continuous batching)

    def serve_start(self, hbm_budget_bytes, max_batch_gates=0):
        self._c(lib().tfhe_serve_start(self._h, int(hbm_budget_bytes), int(max_batch_gates)))

    def serve_submit(self, kind, width, in0, in1, out, rows=0, cols=0) -> int:
        _need_job(1, kind, width, rows, cols, in0, in1, out)
        req = CRequest(kind, width, rows, cols, _dev(in0).value, _dev(in1).value,
                       _dev(out).value)
        rid = ctypes.c_uint64(0)
        self._c(lib().tfhe_serve_submit(self._h, ctypes.byref(req), ctypes.byref(rid)))
        return int(rid.value)

    def serve_poll(self, rid):
        st, lat = ctypes.c_int(0), ctypes.c_double(0)
        self._c(lib().tfhe_serve_poll(self._h, rid, ctypes.byref(st), ctypes.byref(lat)))
        return int(st.value), float(lat.value)

    def serve_wait(self, rid, timeout_ms=60000) -> float:
        lat = ctypes.c_double(0)
        self._c(lib().tfhe_serve_wait(self._h, rid, int(timeout_ms), ctypes.byref(lat)))
        return float(lat.value)

    def serve_cancel(self, rid):
        """Cancel a request that has not completed (TFHEError with TFHE_EBUSY
        when its last level is already on the device, TFHE_EINVAL when it has
        finished or is unknown)."""
        self._c(lib().tfhe_serve_cancel(self._h, rid))

    def serve_stats(self) -> dict:
        info = CServeInfo()
        self._c(lib().tfhe_serve_stats(self._h, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in CServeInfo._fields_}

    def serve_latencies(self) -> np.ndarray:
        n = ctypes.c_size_t(0)
        self._c(lib().tfhe_serve_latencies(self._h, None, 0, ctypes.byref(n)))
        out = np.zeros(n.value, dtype=np.float64)
        if n.value:
            self._c(lib().tfhe_serve_latencies(self._h, ctypes.c_void_p(out.ctypes.data),
                                               n.value, ctypes.byref(n)))
        return out

    def serve_stop(self):
        self._c(lib().tfhe_serve_stop(self._h))


def schedule_info(jobs, policy=1, target=0):
    """Host-only level widths of a job list's schedule (no GPU needed).
    jobs: list of (kind, width, rows, cols, batch).  -> (widths, gates)"""
    arr = (CJob * len(jobs))()
    for k, (kind, width, rows, cols, batch) in enumerate(jobs):
        arr[k] = CJob(kind, width, rows, cols, batch, None, None, None)
    depth, gates = ctypes.c_int32(0), ctypes.c_int64(0)
    _check(lib().tfhe_schedule_info(arr, len(jobs), policy, target, None, 0,
                                    ctypes.byref(depth), ctypes.byref(gates)))
    widths = np.zeros(max(depth.value, 1), dtype=np.int32)
    _check(lib().tfhe_schedule_info(arr, len(jobs), policy, target,
                                    ctypes.c_void_p(widths.ctypes.data), depth.value,
                                    ctypes.byref(depth), ctypes.byref(gates)))
    return widths[:depth.value], int(gates.value)


def serve_select(width, remaining, waited, cap, num_sms, level_ms=None, wave_ms=0.0):
    """Host-only: indices of the requests one serving iteration takes, in
    rank order (tfhe_serve_select; no GPU needed)."""
    w = np.ascontiguousarray(width, dtype=np.int64)
    r = np.ascontiguousarray(remaining, dtype=np.int32)
    t = np.ascontiguousarray(waited, dtype=np.int32)
    if not (len(w) == len(r) == len(t)):
        raise ValueError("width, remaining and waited differ in length")
    lm = None if level_ms is None else np.ascontiguousarray(level_ms, dtype=np.float32)
    if lm is not None and lm.shape != (8,):
        raise ValueError("level_ms holds 8 bucket times")
    out = np.zeros(max(len(w), 1), dtype=np.int32)
    nt = ctypes.c_size_t(0)
    _check(lib().tfhe_serve_select(
        ctypes.c_void_p(w.ctypes.data), ctypes.c_void_p(r.ctypes.data),
        ctypes.c_void_p(t.ctypes.data), len(w), cap, num_sms,
        None if lm is None else ctypes.c_void_p(lm.ctypes.data), wave_ms,
        ctypes.c_void_p(out.ctypes.data), ctypes.byref(nt)))
    return out[:nt.value].copy()


def tc_key_bytes() -> int:
    """Bytes of the tensor-pipe key operand of one CMux step."""
    return int(lib().tfhe_tc_key_bytes())


def tc_digit_bytes(count) -> int:
    """Bytes of the tensor-pipe digit operand scratch for `count` bootstraps."""
    return int(lib().tfhe_tc_digit_bytes(count))


def circuit_info(kind, width, rows=0, cols=0):
    """(bootstrapped gates, depth) of one instance of a circuit."""
    g, d = ctypes.c_int64(0), ctypes.c_int32(0)
    _check(lib().tfhe_circuit_info(kind, width, rows, cols, ctypes.byref(g), ctypes.byref(d)))
    return int(g.value), int(d.value)


def circuit_eval_plain(kind, width, in_bits, n_out, rows=0, cols=0) -> np.ndarray:
    """Host-only: the circuit's netlist evaluated on plaintext bits (uint8
    0/1 input wires in circuit order) -> n_out output bits."""
    inp = np.ascontiguousarray(np.asarray(in_bits, dtype=np.uint8))
    out = np.zeros(n_out, dtype=np.uint8)
    _check(lib().tfhe_circuit_eval_plain(kind, width, rows, cols, _ptr(inp), inp.size,
                                         _ptr(out), n_out))
    return out


# ------------------------------------------------------------- client side

def keygen(params: TFHEParams, s, S, bk_mask, bk_noise, ksk_mask, ksk_noise, stream=None):
    """Device key generation from device draws -> (bk, ksk) int32 tensors."""
    import torch
    p = params
    dev = s.device
    bk = torch.empty((p.n, 2 * p.l, 2, p.N), dtype=torch.int32, device=dev)
    ksk = torch.empty((p.N, p.ks_t, p.ks_digits, p.n + 1), dtype=torch.int32, device=dev)
    cp = CParams.of(p)
    _check(lib().tfhe_keygen(ctypes.byref(cp), _dev(s), _dev(S), _dev(bk_mask), _dev(bk_noise),
                             _dev(ksk_mask), _dev(ksk_noise), _dev(bk), _dev(ksk),
                             _stream(stream)))
    return bk, ksk


def encrypt_bits(params: TFHEParams, s, masks, noise, bits, stream=None):
    """bits uint8 [...]; masks uint32-as-int32 [..., n]; -> int32 [..., 512]."""
    import torch
    out = torch.empty(tuple(bits.shape) + (LWE_STRIDE,), dtype=torch.int32, device=bits.device)
    cp = CParams.of(params)
    _check(lib().tfhe_encrypt_bits(ctypes.byref(cp), _dev(s), _dev(masks), _dev(noise),
                                   _dev(bits, torch.uint8), _dev(out), bits.numel(),
                                   _stream(stream)))
    return out


def phase(params: TFHEParams, s, cts, stream=None):
    """-> int32 tensor of phases (b - <a, s>) with the leading shape of cts."""
    import torch
    count = cts.numel() // LWE_STRIDE
    out = torch.empty(cts.shape[:-1], dtype=torch.int32, device=cts.device)
    cp = CParams.of(params)
    _check(lib().tfhe_phase(ctypes.byref(cp), _dev(s), _dev(cts), _dev(out), count,
                            _stream(stream)))
    return out


def decrypt_bits(params: TFHEParams, s, cts, stream=None):
    return (phase(params, s, cts, stream) > 0).to(dtype=__import__("torch").uint8)


def to_device(a: np.ndarray, device="cuda"):
    """numpy (u)int32/uint8 array -> torch tensor on device (uint32 viewed as int32)."""
    import torch
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)
