"""tfs_topk_noalloc: the top-k for callers that cannot allocate device memory
(a budgeted serving loop, a process whose free device memory belongs to
another framework's allocator, a loop that cannot afford cudaMalloc's
possible device synchronisation).  Its scratch is a fixed device array
inside the library, so it must give exactly what tfs_topk gives, call after
call, and refuse inputs larger than that array serves.

This file is collected last on purpose: a failure here leaves every other
test already run.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_20891_gb300 import build as B

    B.build()
    from paper_2510_20891_gb300 import _lib

    return torch, _lib.lib(), _lib.check


def _both(torch, L, check, v, k):
    """Top-k of device values through the allocating and the non-allocating entry points."""
    N = v.numel()
    kk = min(k, N)
    out = []
    for name in ("tfs_topk", "tfs_topk_noalloc"):
        idx = torch.full((kk,), -7, dtype=torch.int64, device="cuda")
        val = torch.full((kk,), float("nan"), dtype=torch.float32, device="cuda")
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        if name == "tfs_topk":
            check(L.tfs_topk(v.data_ptr(), N, k, idx.data_ptr(), val.data_ptr(), 1, stream))
        else:
            check(L.tfs_topk_noalloc(v.data_ptr(), N, k, idx.data_ptr(), val.data_ptr(), stream))
        torch.cuda.synchronize()
        out.append((idx.cpu().numpy(), val.cpu().numpy()))
    return out


def test_noalloc_topk_matches_allocating_topk_twice(env):
    torch, L, check = env
    g = torch.Generator(device="cuda").manual_seed(11)
    # two calls in a row with different data and sizes: the shared scratch must not leak state
    cases = [(torch.randn(3_000_017, device="cuda", generator=g), 1000),
             ((torch.randint(0, 40, (123_457,), device="cuda", generator=g) * 0.5).float(), 128)]
    cases[1][0][::997] = float("nan")
    for v, k in cases:
        (i0, v0), (i1, v1) = _both(torch, L, check, v, k)
        assert np.array_equal(i0, i1)
        assert np.array_equal(v0, v1, equal_nan=True)
        host = v.cpu().numpy().astype(np.float64)
        nan = np.isnan(host)
        ref = np.lexsort((np.arange(host.size), np.where(nan, 0.0, -host) + 0.0, nan))[: min(k, host.size)]
        assert np.array_equal(i1, ref)


def test_noalloc_topk_rejects_inputs_beyond_its_scratch(env):
    torch, L, check = env
    v = torch.zeros(8, device="cuda")
    idx = torch.zeros(4, dtype=torch.int64, device="cuda")
    val = torch.zeros(4, device="cuda")
    rc = L.tfs_topk_noalloc(v.data_ptr(), (1 << 26) + 1, 4, idx.data_ptr(), val.data_ptr(), None)
    assert rc == -1
    assert b"2^26" in L.tfs_last_error() or b"67108864" in L.tfs_last_error()
    assert L.tfs_topk_noalloc(v.data_ptr(), 8, 0, idx.data_ptr(), val.data_ptr(), None) == -1
