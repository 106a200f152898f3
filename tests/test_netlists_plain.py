"""The CUDA library's circuit netlists evaluated on plaintext bits on the
host (tfhe_circuit_eval_plain, the same gate lists the GPU schedules run):
every circuit kind against Python integer arithmetic, exhaustively at small
widths and on random and edge operands up to 64 bits.  No GPU and no
cryptography: this pins the circuit definitions themselves."""
import numpy as np
import pytest

from paper_2005_01945_gb300 import synth


@pytest.fixture(scope="module")
def api():
    from paper_2005_01945_gb300 import api, build
    build.build()
    return api


def _bits(x, w):
    return [(int(x) >> i) & 1 for i in range(w)]


def _int(bits):
    return sum(int(b) << i for i, b in enumerate(bits))


def _operands(w, n, seed):
    """All pairs for w <= 5; else edge operands (carry and borrow chains)
    and n random pairs."""
    if w <= 5:
        return [(a, b) for a in range(1 << w) for b in range(1 << w)]
    ones, top = (1 << w) - 1, 1 << (w - 1)
    edges = [(ones, 1), (ones, ones), (top, top), (top, ones), (0, ones), (1, ones),
             (top | 1, ones), (ones ^ 1, 3)]
    rng = np.random.default_rng(seed)
    rand = [(int(rng.integers(0, 1 << 62)) & ones, int(rng.integers(0, 1 << 62)) & ones)
            for _ in range(n)]
    return edges + rand


def _eval(api, kind, w, a, b, n_out):
    return _int(api.circuit_eval_plain(kind, w, _bits(a, w) + _bits(b, w), n_out))


ADDERS = ["ADD", "ADD_MAJ", "ADD_NW", "ADD_PREFIX"]
TRUNC_MULS = ["MUL", "MUL_TREE", "MUL_TREE_MAJ", "MUL_DADDA"]
FULL_MULS = ["MUL_FULL", "MUL_KARATSUBA"]


@pytest.mark.parametrize("name", ADDERS)
@pytest.mark.parametrize("w", [1, 2, 3, 4, 5, 7, 8, 13, 16, 31, 32, 33, 64])
def test_adders(api, name, w):
    kind = getattr(api, name)
    for a, b in _operands(w, 24, 100 + w):
        assert _eval(api, kind, w, a, b, w) == (a + b) % (1 << w), (name, w, a, b)


@pytest.mark.parametrize("name", TRUNC_MULS)
@pytest.mark.parametrize("w", [1, 2, 3, 4, 5, 6, 9, 16, 17, 32, 64])
def test_truncated_multipliers(api, name, w):
    kind = getattr(api, name)
    for a, b in _operands(w, 12, 200 + w):
        assert _eval(api, kind, w, a, b, w) == (a * b) % (1 << w), (name, w, a, b)


@pytest.mark.parametrize("name", FULL_MULS)
@pytest.mark.parametrize("w", [2, 3, 4, 5, 8, 9, 16, 17, 32, 64])
def test_full_products(api, name, w):
    kind = getattr(api, name)
    for a, b in _operands(w, 8, 300 + w):
        assert _eval(api, kind, w, a, b, 2 * w) == a * b, (name, w, a, b)


@pytest.mark.parametrize("rows,cols,w", [(1, 1, 1), (2, 3, 4), (3, 5, 6), (4, 4, 16)])
def test_matvec(api, rows, cols, w):
    rng = np.random.default_rng(rows * 100 + cols * 10 + w)
    for _ in range(6):
        M = rng.integers(0, 1 << w, size=(rows, cols), dtype=np.uint64)
        v = rng.integers(0, 1 << w, size=cols, dtype=np.uint64)
        bits = [bit for r in range(rows) for c in range(cols) for bit in _bits(M[r, c], w)]
        bits += [bit for c in range(cols) for bit in _bits(v[c], w)]
        out = api.circuit_eval_plain(api.MATVEC, w, bits, rows * w, rows, cols)
        for r in range(rows):
            want = sum(int(M[r, c]) * int(v[c]) for c in range(cols)) % (1 << w)
            assert _int(out[r * w:(r + 1) * w]) == want


def test_single_gates_match_truth_tables(api):
    """GATE circuits (opcode in `width`) against the golden truth tables."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "gate_truth_tables.txt")
    tab = {}
    for line in open(path):
        f = line.split("#")[0].split()
        if len(f) == 5:
            tab[f[0]] = [int(x) for x in f[1:]]
    for name, row in tab.items():
        op = getattr(api, name)
        got = [int(api.circuit_eval_plain(api.GATE, op, [a, b], 1)[0])
               for a, b in ((0, 0), (0, 1), (1, 0), (1, 1))]
        assert got == row, name


def test_rejects_bad_counts_and_kinds(api):
    with pytest.raises(api.TFHEError):
        api.circuit_eval_plain(api.ADD, 4, [0] * 7, 4)
    with pytest.raises(api.TFHEError):
        api.circuit_eval_plain(api.ADD, 4, [0] * 8, 5)
    with pytest.raises(api.TFHEError):
        api.circuit_eval_plain(99, 4, [0] * 8, 4)


def test_documented_gate_counts_and_depths(api):
    """The counts and depths the header states, at every width 1..64:
    ripple adder 5w - 6 gates in 2w - 2 levels (w = 1: one XOR), majority
    adder 3w - 2 gates in w levels, number-wise adder w^2 gates in w levels,
    prefix adder ceil(log2(w - 1)) + 2 levels (w >= 3); width 65 is
    refused."""
    import math
    for w in range(1, 65):
        assert api.circuit_info(api.ADD, w) == ((5 * w - 6, 2 * w - 2) if w > 1 else (1, 1))
        if w > 1:
            assert api.circuit_info(api.ADD_MAJ, w) == (3 * w - 2, w)
        assert api.circuit_info(api.ADD_NW, w) == (w * w, w)
        if w >= 3:
            assert api.circuit_info(api.ADD_PREFIX, w)[1] == math.ceil(math.log2(w - 1)) + 2
    for kind in (api.ADD, api.MUL, api.ADD_PREFIX, api.MUL_DADDA, api.MUL_FULL):
        with pytest.raises(api.TFHEError):
            api.circuit_info(kind, 65)
