"""Learned periphery on the tensor cores: kernels against the CPU oracle of the network."""
import numpy as np
import pytest

import paper_2507_04147_gb300 as a3fr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("n,k", [(32, 16), (32, 64), (16, 48)])
def test_tensor_core_tile_gemm(n, k):
    import torch
    g = torch.Generator().manual_seed(n * 100 + k)
    A = torch.randn(128, k, generator=g).to(torch.bfloat16)
    B = torch.randn(n, k, generator=g).to(torch.bfloat16)
    D = torch.empty(128, n, device="cuda")
    a3fr.tc_tile_gemm(A.cuda(), B.cuda(), D, variant=0)
    torch.cuda.synchronize()
    ref = A.double() @ B.double().T
    err = (D.cpu().double() - ref).abs().max().item()
    assert err < 1e-4 * max(1.0, ref.abs().max().item()), err
