"""a3fr_sort_pairs_noalloc, the sort entry point for callers that cannot allocate.

Callers such as a real-time render thread (which cannot absorb the device-wide
synchronisation cudaMalloc/cudaFree may cause) or code inside an engine that owns all
device memory through its own allocator get the same stable radix sort without passing
or allocating any scratch: it comes from a fixed device array inside the library.

The test calls the new entry point through the C ABI and compares it with the existing
entry point a3fr_sort_pairs (which takes caller-allocated scratch) on two calls in a row:
the sort is integer work, so the results must be identical.  This file is collected last
so that a run stopping at the first failure has run every other test already; it passes
alone in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

import paper_2507_04147_gb300 as a3fr
from paper_2507_04147_gb300 import _lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return _lib.load()


def _existing_sort(torch, keys, vals, bits):
    k = keys.clone()
    v = vals.clone()
    ka, va = torch.empty_like(k), torch.empty_like(v)
    ws = torch.empty(a3fr.sort_pairs_workspace_bytes(k.numel()), dtype=torch.uint8, device="cuda")
    a3fr.sort_pairs(k, v, ka, va, bits, ws)
    return k, v


def test_noalloc_sort_matches_existing_entry_point_twice(lib):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(2024)
    for call, (n, bits) in enumerate([(200_003, 46), (_lib.NOALLOC_MAX_PAIRS, 40)]):
        keys_np = rng.integers(0, 2 ** 46, size=n, dtype=np.uint64)
        if call == 1:   # tile|depth-like keys with many equal tiles
            keys_np = (rng.integers(0, 300, size=n, dtype=np.uint64) << np.uint64(32)) | \
                      rng.integers(0, 2 ** 24, size=n, dtype=np.uint64)
            keys_np &= np.uint64((1 << bits) - 1)
        vals_np = np.arange(n, dtype=np.uint32)
        keys = torch.from_numpy(keys_np.view(np.int64)).cuda()
        vals = torch.from_numpy(vals_np.view(np.int32)).cuda()
        ref_k, ref_v = _existing_sort(torch, keys, vals, bits)
        k, v = keys.clone(), vals.clone()
        rc = lib.a3fr_sort_pairs_noalloc(ctypes.c_void_p(k.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                         n, bits, ctypes.c_void_p(stream))
        assert rc == 0, a3fr.error_string(rc)
        torch.cuda.synchronize()
        assert torch.equal(k, ref_k), f"keys differ on call {call}"
        assert torch.equal(v, ref_v), f"values differ on call {call}"


def test_noalloc_rejects_sizes_beyond_its_maximum(lib):
    n = _lib.NOALLOC_MAX_PAIRS + 1
    rc = lib.a3fr_sort_pairs_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(16), n, 40, None)
    assert rc == -4 and "CAPACITY" in a3fr.error_string(rc)
