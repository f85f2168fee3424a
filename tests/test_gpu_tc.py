"""tcgen05 contraction (afqmc_contract) against a float64 reference.

C = alpha A B^T with BF16 or TF32 operands and FP32 accumulation.  The
reference multiplies the operands after rounding them to the input type, in
float64, so the only difference left is FP32 accumulation (relative
Frobenius error ~ 1e-6 for these K).
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
    import __graft_entry__

    __graft_entry__.build()
    import paper_1711_02242_gb300 as pkg

    return torch, pkg


def contract(torch, pkg, A, B, k, alpha=1.0, tf32=False):
    m, n = A.shape[0], B.shape[0]
    C = torch.full((m, n + 3), float("nan"), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = pkg.lib().afqmc_contract(1 if tf32 else 0, m, n, k, ctypes.c_void_p(A.data_ptr()),
                                  A.stride(0), ctypes.c_void_p(B.data_ptr()), B.stride(0),
                                  ctypes.c_float(alpha), ctypes.c_void_p(C.data_ptr()), C.stride(0),
                                  ctypes.c_void_p(st.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    pkg._check(rc)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return C[:, :n]


@pytest.mark.parametrize("m,n,k,pitch", [
    (128, 256, 64, 64),      # one tile, one stage
    (256, 512, 1856, 1856),  # many stages, ring wraps
    (200, 300, 136, 144),    # ragged M, N and K (pitch > k)
    (1024, 2000, 1800, 1856),  # V-contraction-like shape
])
def test_bf16_contraction(env, m, n, k, pitch):
    torch, pkg = env
    g = torch.Generator(device="cuda").manual_seed(m + n + k)
    A = torch.randn((m, pitch), generator=g, device="cuda").to(torch.bfloat16)
    B = torch.randn((n, pitch), generator=g, device="cuda").to(torch.bfloat16)
    C = contract(torch, pkg, A, B, k, alpha=2.0)
    ref = 2.0 * (A[:, :k].double() @ B[:, :k].double().T)
    err = torch.linalg.norm(C.double() - ref) / torch.linalg.norm(ref)
    assert err < 1e-5, float(err)


@pytest.mark.parametrize("m,n,k,pitch", [(128, 256, 32, 32), (300, 500, 520, 524)])
def test_tf32_contraction(env, m, n, k, pitch):
    torch, pkg = env
    g = torch.Generator(device="cuda").manual_seed(7 + m)
    A = torch.randn((m, pitch), generator=g, device="cuda", dtype=torch.float32)
    B = torch.randn((n, pitch), generator=g, device="cuda", dtype=torch.float32)
    C = contract(torch, pkg, A, B, k, tf32=True)
    ref = A[:, :k].double() @ B[:, :k].double().T
    err = torch.linalg.norm(C.double() - ref) / torch.linalg.norm(ref)
    assert err < 2e-3, float(err)
    # the TF32 rounding of the inputs is the only loss: much better than BF16
    Ab, Bb = A[:, :k].bfloat16().double(), B[:, :k].bfloat16().double()
    err_b = torch.linalg.norm(Ab @ Bb.T - ref) / torch.linalg.norm(ref)
    assert err < 0.5 * err_b
