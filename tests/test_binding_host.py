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
