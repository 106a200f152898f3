"""The ctypes binding agrees with the C header it marshals for, checked on
the CPU without loading a GPU: every function the header declares has a
binding entry with the same number of parameters, each of the size and
kind (pointer, integer, floating point) the header gives it, and the same
return type; the structures passed by pointer have the header's fields in
the header's order and sizes; and the status codes, circuit kinds and
option numbers the binding uses are the header's values."""
import ctypes
import os
import re

import pytest

from paper_2005_01945_gb300 import api

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C scalar types of the header -> (size in bytes, kind)
C_SCALARS = {
    "int": (4, "int"), "int32_t": (4, "int"), "uint32_t": (4, "int"),
    "int64_t": (8, "int"), "uint64_t": (8, "int"), "size_t": (8, "int"),
    "float": (4, "float"), "double": (8, "float"),
}


def _header():
    src = open(os.path.join(ROOT, "include", "tfhe_gb.h")).read()
    return re.sub(r"/\*.*?\*/", "", src, flags=re.S)


def _declarations():
    """name -> (return type, [parameter declarations])"""
    out = {}
    for m in re.finditer(r"\b(int|size_t|void)\s+(tfhe_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", _header()):
        params = [q.strip() for q in m.group(3).split(",") if q.strip()]
        if params == ["void"]:
            params = []
        out[m.group(2)] = (m.group(1), params)
    return out


def _c_param(decl):
    """(size, kind) of one C parameter declaration."""
    if "*" in decl:
        return 8, "ptr"
    words = decl.replace("const", " ").split()
    return C_SCALARS[words[0]]


def _ctypes_kind(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and \
            isinstance(t._type_, type):
        return ctypes.sizeof(t), "ptr"
    if t in (ctypes.c_float, ctypes.c_double):
        return ctypes.sizeof(t), "float"
    return ctypes.sizeof(t), "int"


def test_every_declared_function_is_bound():
    decl = _declarations()
    assert len(decl) >= 30          # the parse found the declarations
    assert set(decl) == set(api.EXPORTS), set(decl) ^ set(api.EXPORTS)


@pytest.mark.parametrize("name", sorted(_declarations()))
def test_function_signature_matches(name):
    ret, params = _declarations()[name]
    restype, argtypes = api.EXPORTS[name]
    assert len(argtypes) == len(params), (name, params)
    for k, (decl, t) in enumerate(zip(params, argtypes)):
        assert _ctypes_kind(t) == _c_param(decl), (name, k, decl, t)
    want_ret = {"int": ctypes.c_int, "size_t": ctypes.c_size_t, "void": None}[ret]
    assert restype is want_ret, (name, ret, restype)


def _struct_fields(name):
    m = re.search(r"typedef struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", _header(), flags=re.S)
    assert m, name
    fields = []
    for stmt in m.group(1).split(";"):
        stmt = stmt.strip()
        if not stmt:
            continue
        stmt = stmt.replace("const", " ").strip()
        base = stmt.split()[0]
        for var in stmt[len(base):].split(","):
            var = var.strip()
            ptr = var.startswith("*")
            fields.append((var.lstrip("*").strip(), 8 if ptr else C_SCALARS[base][0]))
    return fields


@pytest.mark.parametrize("cname,pyname", [("tfhe_params", "CParams"), ("tfhe_job", "CJob"),
                                          ("tfhe_request", "CRequest"),
                                          ("tfhe_serve_info", "CServeInfo")])
def test_struct_layout_matches(cname, pyname):
    want = _struct_fields(cname)
    cls = getattr(api, pyname)
    got = [(f, ctypes.sizeof(t)) for f, t in cls._fields_]
    assert got == want, (cname, got, want)


def _enum_values(name):
    m = re.search(r"typedef enum\s*\{([^{}]*)\}\s*" + name + r"\s*;", _header(), flags=re.S)
    assert m, name
    vals = {}
    for item in m.group(1).split(","):
        item = item.strip()
        if item:
            k, v = (s.strip() for s in item.split("="))
            vals[k] = int(v)
    return vals


def test_status_codes_match():
    vals = _enum_values("tfhe_status")
    assert {v: k for k, v in vals.items()} == api._STATUS


def test_circuit_kinds_and_options_match():
    kinds = _enum_values("tfhe_circuit")
    for cname, pyname in [("GATE", "GATE"), ("ADD", "ADD"), ("MUL", "MUL"),
                          ("MATVEC", "MATVEC"), ("ADD_MAJ", "ADD_MAJ"), ("ADD_NW", "ADD_NW"),
                          ("MUL_TREE", "MUL_TREE"), ("MUL_FULL", "MUL_FULL"),
                          ("MUL_KARATSUBA", "MUL_KARATSUBA"), ("MUL_TREE_MAJ", "MUL_TREE_MAJ"),
                          ("ADD_PREFIX", "ADD_PREFIX"), ("MUL_DADDA", "MUL_DADDA")]:
        assert kinds["TFHE_CIRCUIT_" + cname] == getattr(api, pyname), cname
    assert len(kinds) == 12
    opts = _enum_values("tfhe_option")
    assert {k[len("TFHE_OPT_"):]: v for k, v in opts.items()} == \
        {k[len("OPT_"):]: getattr(api, k) for k in dir(api) if k.startswith("OPT_")}
    gates = _enum_values("tfhe_gate")
    assert [gates["TFHE_" + g] for g in api.GATE_NAMES] == list(range(len(api.GATE_NAMES)))
    sched = _enum_values("tfhe_schedule")
    assert (sched["TFHE_SCHED_ASAP"], sched["TFHE_SCHED_BALANCED"]) == \
        (api.SCHED_ASAP, api.SCHED_BALANCED)
