"""The CMux step's negacyclic products on the tensor pipe (tcgen05, limb-split
bf16 operands, exact fp32 sums), the measured alternative to the NTT:
every output word equals the oracle's schoolbook products, through the C
ABI, with extreme digits and key words among the inputs and inputs that
span two 128-bootstrap tiles and all 8 column tiles."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_tc_products_bit_exact(orc):
    import torch
    from paper_2005_01945_gb300 import api, build, synth
    build.build()
    count = 256
    g = synth._gen(5, "tc_products")
    dig = g.integers(-512, 512, size=(count, 4, 1024), dtype=np.int64).astype(np.int32)
    dig[0] = -512                      # the most negative digit everywhere
    dig[1] = 511                       # the most positive
    dig[2] = 0
    dig[3, :, ::2], dig[3, :, 1::2] = -512, 511
    bk = g.integers(0, 1 << 32, size=(4, 2, 1024), dtype=np.uint64).astype(np.uint32)
    bk[0, 0, :8] = [0, 1, 0x7F, 0x80, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFF, 0x80808080]
    bk[3, 1, -4:] = 0xFFFFFFFF
    ctx = api.Context(synth.TFHEParams())
    try:
        key_ops = torch.empty(api.tc_key_bytes(), dtype=torch.uint8, device="cuda")
        digit_ops = torch.empty(api.tc_digit_bytes(count), dtype=torch.uint8, device="cuda")
        out = torch.full((count, 2, 1024), -1, dtype=torch.int32, device="cuda")
        ctx.tc_prepare_key(api.to_device(bk), key_ops)
        ctx.cmux_products_tc(api.to_device(dig), key_ops, digit_ops, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        assert ctx.status() == 0
        for m in range(count):
            for p in range(2):
                want = np.zeros(1024, dtype=np.uint32)
                for r in range(4):
                    want += orc.negacyclic_mul(dig[m, r], bk[r, p])
                assert np.array_equal(got[m, p], want), (m, p)
    finally:
        ctx.close()


def test_tc_products_refuse_bad_counts():
    import torch
    from paper_2005_01945_gb300 import api, build, synth
    build.build()
    ctx = api.Context(synth.TFHEParams())
    try:
        key_ops = torch.empty(api.tc_key_bytes(), dtype=torch.uint8, device="cuda")
        dig = torch.zeros((100, 4, 1024), dtype=torch.int32, device="cuda")
        ops = torch.empty(api.tc_digit_bytes(100), dtype=torch.uint8, device="cuda")
        out = torch.empty((100, 2, 1024), dtype=torch.int32, device="cuda")
        with pytest.raises(api.TFHEError) as e:
            ctx.cmux_products_tc(dig, key_ops, ops, out)
        assert e.value.code == -1 and "multiple of 128" in str(e.value)
    finally:
        ctx.close()
