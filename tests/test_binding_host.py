"""The Python binding fails loudly instead of falling back to the CPU: a
missing library, a host without a GPU and host tensors are all refused
before any computation.  No GPU is used."""
import numpy as np
import pytest
import torch

from paper_2005_01945_gb300 import synth


@pytest.fixture(scope="module")
def api():
    from paper_2005_01945_gb300 import api, build
    build.build()
    return api


def test_missing_library_raises(api, monkeypatch, tmp_path):
    monkeypatch.setattr(api, "LIB_PATH", str(tmp_path / "libtfhe_gb.so"))
    monkeypatch.setattr(api, "_lib", None)
    with pytest.raises(RuntimeError, match="is missing"):
        api.lib()


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU host")
def test_context_without_gpu_is_an_error(api):
    with pytest.raises(api.TFHEError) as err:
        api.Context(synth.TFHEParams())
    assert err.value.code == -3                      # TFHE_ECUDA


def test_host_tensors_are_refused(api):
    p = synth.TFHEParams(n=8, N=32)
    kd = synth.key_draws(p, 5)
    host = lambda a: torch.from_numpy(np.ascontiguousarray(
        a.view(np.int32) if a.dtype == np.uint32 else a))
    with pytest.raises(TypeError, match="CUDA tensor"):
        api.keygen(p, host(kd.s), host(kd.S), host(kd.bk_mask), host(kd.bk_noise),
                   host(kd.ksk_mask), host(kd.ksk_noise))
    cd = synth.ct_draws(p, (4,), 5, "host")
    with pytest.raises(TypeError, match="CUDA tensor"):
        api.encrypt_bits(p, host(kd.s), host(cd.mask), host(cd.noise),
                         torch.zeros(4, dtype=torch.uint8))
    with pytest.raises(TypeError, match="CUDA tensor"):
        api._dev(np.zeros(4, np.int32))


def test_non_contiguous_host_arrays_are_refused(api):
    a = np.zeros((4, 4), np.int32)[:, ::2]
    with pytest.raises(ValueError, match="contiguous"):
        api._ptr(a)
    assert api._ptr(None) is None
    assert api._ptr(np.zeros(4, np.int32)).value is not None


@pytest.mark.parametrize("kind_name,w,rows,cols", [
    ("GATE", 3, 0, 0), ("ADD", 8, 0, 0), ("ADD_MAJ", 5, 0, 0), ("ADD_NW", 4, 0, 0),
    ("ADD_PREFIX", 9, 0, 0), ("MUL", 6, 0, 0), ("MUL_TREE", 5, 0, 0), ("MUL_TREE_MAJ", 7, 0, 0),
    ("MUL_DADDA", 8, 0, 0), ("MUL_FULL", 4, 0, 0), ("MUL_KARATSUBA", 9, 0, 0),
    ("MATVEC", 3, 2, 5)])
def test_job_rows_match_the_library_netlists(api, kind_name, w, rows, cols):
    """The binding's per-instance row counts (used to refuse short buffers)
    equal the input and output wire counts of the library's own netlist:
    the plain evaluator accepts exactly those counts and refuses one more."""
    kind = getattr(api, kind_name)
    r0, r1, ro = api.job_rows(kind, w, rows, cols)
    out = api.circuit_eval_plain(kind, w, [0] * (r0 + r1), ro, rows, cols)
    assert out.shape == (ro,)
    with pytest.raises(api.TFHEError):
        api.circuit_eval_plain(kind, w, [0] * (r0 + r1 + 1), ro, rows, cols)
    with pytest.raises(api.TFHEError):
        api.circuit_eval_plain(kind, w, [0] * (r0 + r1), ro + 1, rows, cols)


def test_short_buffers_are_refused_before_any_launch(api):
    """A buffer smaller than its job needs raises TFHE_EINVAL in the binding
    (the library trusts the sizes it is given)."""
    S = api.LWE_STRIDE
    z = lambda *shape: torch.zeros(shape, dtype=torch.int32)
    api._need_job(4, api.ADD, 8, 0, 0, z(4, 8, S), z(4, 8, S), z(4, 8, S))
    api._need_job(0, api.ADD, 8, 0, 0, z(0), z(0), z(0))            # empty batch
    for args in ((z(3, 8, S), z(4, 8, S), z(4, 8, S)),
                 (z(4, 8, S), z(4, 8, S - 1), z(4, 8, S)),
                 (z(4, 8, S), z(4, 8, S), z(4, 7, S))):
        with pytest.raises(api.TFHEError) as err:
            api._need_job(4, api.ADD, 8, 0, 0, *args)
        assert err.value.code == -1
    with pytest.raises(api.TFHEError):                               # 2w output rows
        api._need_job(1, api.MUL_FULL, 8, 0, 0, z(8, S), z(8, S), z(8, S))
    api._need_job(1, api.MUL_FULL, 8, 0, 0, z(8, S), z(8, S), z(16, S))
    with pytest.raises(api.TFHEError):                               # M is rows x cols x w
        api._need_job(1, api.MATVEC, 4, 3, 2, z(2, 2, 4, S), z(2, 4, S), z(3, 4, S))
    with pytest.raises(api.TFHEError):
        api._need(z(10, api.BIG_STRIDE - 1), 10, "big", api.BIG_STRIDE)
