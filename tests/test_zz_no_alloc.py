"""mwcg_dot_noalloc: the dot product for callers that must not allocate device memory.

Such callers cannot use mwcg_dot, which allocates and frees its scratch on
every call (and cudaFree synchronises the whole device).  The allocation-free
entry point keeps its scratch in a fixed array inside the library; it must
return exactly what mwcg_dot returns, call after call, because every call
reuses (and must correctly reset) that array.  This file runs last so that a
failure here stops a run only after every other test has run.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_13536_gb300 import _capi, build, solver
    build.build()
    return torch, _capi.load(), solver


def _noalloc_dot(torch, L, arith_id, u, v, G):
    w = u.shape[0]
    out = torch.full((w,), np.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = L.mwcg_dot_noalloc(arith_id, u.shape[1], ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                            int(G), ctypes.c_void_p(stream.cuda_stream), ctypes.c_void_p(out.data_ptr()))
    stream.synchronize()
    return rc, out.cpu().numpy()


def test_noalloc_dot_equals_allocating_dot_on_consecutive_calls(env):
    torch, L, mw = env
    rng = np.random.default_rng(21)
    for call in range(2):                                   # two calls in a row reuse the same scratch
        for arith in ("qtw", "dw", "qdw", "tw", "fp64", "qw", "qqw", "qqw_nn"):
            a = mw.arith_id(arith)
            w = mw.words(arith)
            for n, G in ((70001, 152), (5000, 1024), (257, 3), (1, 1)):
                scale = np.array([1.0, 1e-17, 1e-34, 1e-51][:w])[:, None]
                u = torch.as_tensor(rng.standard_normal((w, n)) * scale, device="cuda")
                v = torch.as_tensor(rng.standard_normal((w, n)) * scale, device="cuda")
                rc, got = _noalloc_dot(torch, L, a, u, v, G)
                assert rc == 0, L.mwcg_last_error()
                ref = mw.dot(arith, u, v, G)                   # the allocating entry point
                assert np.array_equal(got.view(np.uint64), np.asarray(ref).view(np.uint64)), (call, arith, n, G)


def test_noalloc_dot_fp32_words(env):
    """QQF and QF: the packed FP32 layout in, one FP32 word per double out,
    the same bits as mwcg_dot."""
    torch, L, mw = env
    from paper_2510_13536_gb300.solver import _pack
    rng = np.random.default_rng(22)
    for call in range(2):
        for arith in ("qqf", "qf"):
            for n, G in ((70001, 152), (5000, 1024), (257, 3), (1, 1), (0, 5)):
                w32 = np.empty((2, 4, n), dtype=np.float32)
                for j in range(2):
                    w32[j, 0] = rng.standard_normal(n).astype(np.float32)
                    for k in range(1, 4):
                        w32[j, k] = (w32[j, k - 1] * np.float32(2.0 ** -24) * rng.uniform(-1, 1, n)).astype(np.float32)
                u32, v32 = (torch.as_tensor(w32[j], device="cuda") for j in range(2))
                u, v = _pack(u32, n), _pack(v32, n)
                out = torch.full((4,), np.nan, dtype=torch.float64, device="cuda")
                stream = torch.cuda.current_stream()
                rc = L.mwcg_dot_noalloc(mw.arith_id(arith), n, ctypes.c_void_p(u.data_ptr()),
                                        ctypes.c_void_p(v.data_ptr()), G, ctypes.c_void_p(stream.cuda_stream),
                                        ctypes.c_void_p(out.data_ptr()))
                stream.synchronize()
                assert rc == 0, L.mwcg_last_error()
                got = out.cpu().numpy()
                ref = np.asarray(mw.dot(arith, u32, v32, G), dtype=np.float64)
                assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), (call, arith, n, G, got, ref)


def test_noalloc_dot_rejects_oversized_grid(env):
    torch, L, mw = env
    u = torch.zeros((3, 10), dtype=torch.float64, device="cuda")
    rc, _ = _noalloc_dot(torch, L, 4, u, u, 1025)
    assert rc == -1
    assert b"1..1024" in L.mwcg_last_error()
    assert L.mwcg_dot_noalloc(12, 10, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                              1, None, ctypes.c_void_p(u.data_ptr())) == -1     # no arithmetic 12
    assert b"unknown arithmetic" in L.mwcg_last_error()
