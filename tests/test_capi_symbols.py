"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/tfhe_gb.h declares (no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tfhe_gb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tfhe_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tfhe_bootstrap_gates", "tfhe_add_n", "tfhe_mul_n", "tfhe_matvec",
                     "tfhe_ctx_create", "tfhe_ctx_set_keys", "tfhe_ctx_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2005_01945_gb300 import api, build
    build.build()
    L = ctypes.CDLL(api.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    # the Python binding covers the same names
    assert set(api.EXPORTS) <= set(declared_functions())


def test_invalid_params_rejected_without_gpu():
    from paper_2005_01945_gb300 import api
    L = api.lib()
    bad = api.CParams(500, 2048, 1, 2, 10, 8, 2)   # unsupported ring degree
    h = ctypes.c_void_p()
    assert L.tfhe_ctx_create(ctypes.byref(bad), 0, ctypes.byref(h)) == -1
    assert not h.value


def declared_arity():
    src = open(os.path.join(ROOT, "include", "tfhe_gb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for name, args in re.findall(r"\b(tfhe_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", src):
        args = args.strip()
        out[name] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_signatures_match_header():
    from paper_2005_01945_gb300 import api
    arity = declared_arity()
    for name, (_, argtypes) in api.EXPORTS.items():
        assert len(argtypes) == arity[name], (name, len(argtypes), arity[name])
