"""The onesweep radix sort through the C ABI against a stable library sort (bit-exact)."""
import numpy as np
import pytest

import paper_2507_04147_gb300 as a3fr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def gpu_sort(keys, vals, key_bits):
    import torch
    n = len(keys)
    k = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    v = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    ka = torch.empty_like(k)
    va = torch.empty_like(v)
    ws = torch.empty(a3fr.sort_pairs_workspace_bytes(max(n, 1)), dtype=torch.uint8, device="cuda")
    a3fr.sort_pairs(k, v, ka, va, key_bits, ws)
    torch.cuda.synchronize()
    return k.cpu().numpy().view(np.uint64), v.cpu().numpy().view(np.uint32)


def reference(keys, vals, key_bits):
    mask = np.uint64((1 << key_bits) - 1) if key_bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    order = np.argsort(keys & mask, kind="stable")
    return keys[order], vals[order]


CASES = [
    ("random46", 1_000_003, 46),
    ("random64", 300_000, 64),
    ("random40", 3840 * 3 + 17, 40),
    ("equal", 50_000, 46),
    ("presorted", 200_000, 46),
    ("reversed", 200_000, 46),
    ("fewdigits", 500_000, 46),
]


@pytest.mark.parametrize("kind,n,bits", CASES)
def test_sort_matches_stable_sort(kind, n, bits):
    rng = np.random.default_rng(n)
    if kind.startswith("random"):
        keys = rng.integers(0, 2 ** 63, size=n, dtype=np.uint64) & np.uint64((1 << bits) - 1 if bits < 64 else 2 ** 64 - 1)
        if bits == 64:
            keys = rng.integers(0, 2 ** 63, size=n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=n, dtype=np.uint64)
    elif kind == "equal":
        keys = np.full(n, 0x123456789A, dtype=np.uint64)
    elif kind == "presorted":
        keys = np.sort(rng.integers(0, 2 ** 46, size=n, dtype=np.uint64))
    elif kind == "reversed":
        keys = np.sort(rng.integers(0, 2 ** 46, size=n, dtype=np.uint64))[::-1].copy()
    else:   # tile|depth-like keys: few tiles, depths with few distinct exponents
        tiles = rng.integers(0, 12800, size=n, dtype=np.uint64)
        depth = rng.uniform(2.0, 6.0, size=n).astype(np.float32).view(np.uint32).astype(np.uint64)
        keys = (tiles << np.uint64(32)) | depth
    vals = np.arange(n, dtype=np.uint32)
    gk, gv = gpu_sort(keys, vals, bits)
    rk, rv = reference(keys, vals, bits)
    assert np.array_equal(gk, rk)
    assert np.array_equal(gv, rv)


@pytest.mark.parametrize("n", [1, 2, 3, 31, 255, 256, 257, 3839, 3840, 3841, 4095, 4097, 65535, 65537])
def test_sort_edge_sizes(n):
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 2 ** 40, size=n, dtype=np.uint64)
    vals = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    gk, gv = gpu_sort(keys, vals, 40)
    rk, rv = reference(keys, vals, 40)
    assert np.array_equal(gk, rk) and np.array_equal(gv, rv)


def test_sort_only_low_bits_compared():
    rng = np.random.default_rng(7)
    n = 10_000
    keys = rng.integers(0, 2 ** 63, size=n, dtype=np.uint64)
    vals = np.arange(n, dtype=np.uint32)
    gk, gv = gpu_sort(keys, vals, 16)
    rk, rv = reference(keys, vals, 16)
    assert np.array_equal(gk, rk) and np.array_equal(gv, rv)
