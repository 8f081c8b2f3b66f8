"""GPU: the tensor-core operand layouts (A in tensor memory, B as no-swizzle
K-major core matrices in shared memory) give D = A B^T."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,K", [(128, 16), (128, 128), (16, 128), (64, 32)])
def test_umma_probe(N, K):
    import torch
    from paper_2402_17248_gb300 import bl
    g = torch.Generator().manual_seed(N * 1000 + K)
    A = torch.randn(128, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    want = (A.double() @ B.double().T).numpy()
    Ad, Bd = A.cuda(), B.cuda()
    D = torch.zeros(128, N, dtype=torch.float32, device="cuda")
    results = {}
    for name, (ks, ns, lbo, sbo) in {
        "lbo=K": (128, (K // 8) * 128, 128, (K // 8) * 128),
        "lbo=N": (128, (K // 8) * 128, (K // 8) * 128, 128),
    }.items():
        D.zero_()
        assert bl.bl_debug_umma_probe(Ad, Bd, D, N, K, ks, ns, lbo, sbo) == 0
        torch.cuda.synchronize()
        results[name] = float(np.max(np.abs(D.cpu().double().numpy() - want)))
    bl.bl_poll_device_errors()
    print("umma probe max abs error by descriptor reading:", results)
    assert results["lbo=K"] < 1e-3 * np.max(np.abs(want))
