"""Host logic of the Python binding that needs no GPU: the packing of QQF's
four FP32 words into the C ABI's two 8-byte slots per element (slot k of
element i, at k*n + i, holds words 2k and 2k+1, word 2k at the lower address)."""
import numpy as np
import torch

from paper_2510_13536_gb300 import _capi, solver


import pytest


@pytest.mark.parametrize("n", [1, 2, 7])
def test_qqf_slot_layout_and_round_trip(n):
    x = torch.arange(4 * n, dtype=torch.float32).reshape(4, n) * 0.5 - 3.0
    p = solver._pack(x, n)
    assert p.dtype == torch.float64 and p.shape == (2, n) and p.is_contiguous()
    f = p.view(torch.float32).reshape(-1)
    for k in range(2):
        for i in range(n):
            assert f[2 * (k * n + i)] == x[2 * k, i] and f[2 * (k * n + i) + 1] == x[2 * k + 1, i]
    assert torch.equal(solver._unpack(p, n), x)


@pytest.mark.parametrize("n", [1, 11])
def test_numpy_and_torch_packing_agree(n):
    rng = np.random.default_rng(3)
    x = rng.standard_normal((4, n)).astype(np.float32)
    pt = solver._pack(torch.as_tensor(x), n).numpy()
    pn = solver._pack_np(x, n)
    assert np.array_equal(pt.view(np.uint64), pn.view(np.uint64))
    assert np.array_equal(solver._unpack_np(pn, n), x)


def test_abi_conversion_per_arithmetic():
    n = 5
    for name in ("qqf", "qf"):
        a = _capi.ARITH[name]
        assert _capi.WORDS[a] == 4 and _capi.SLOTS[a] == 2 and a in _capi.FP32_WORDS
    q = _capi.ARITH["qqf"]
    x = torch.ones((4, n), dtype=torch.float32)
    assert solver._to_abi(q, x, n).shape == (2, n)
    assert solver._from_abi(q, solver._to_abi(q, x, n), n).dtype == torch.float32
    for name, a in _capi.ARITH.items():
        if a in _capi.FP32_WORDS:
            continue
        assert _capi.SLOTS[a] == _capi.WORDS[a]
        y = torch.ones((_capi.WORDS[a], n), dtype=torch.float64)
        assert solver._to_abi(a, y, n).data_ptr() == y.data_ptr()       # no copy for FP64 words
        assert solver._from_abi(a, y, n) is y


def test_empty_vectors():
    assert solver._pack(torch.zeros((4, 0), dtype=torch.float32), 0).shape == (2, 0)
    assert solver._unpack(torch.zeros((2, 0), dtype=torch.float64), 0).shape == (4, 0)
    assert solver._pack_np(np.zeros((4, 0), dtype=np.float32), 0).shape == (2, 0)
    assert solver._unpack_np(np.zeros((2, 0)), 0).shape == (4, 0)
