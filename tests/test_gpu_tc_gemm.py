"""The tcgen05 bf16 GEMM against a float64 product of the same bf16 inputs (GPU)."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1004_0024_gb300 import ising
    return torch, ising


def _gemm(env, A, B, bias=None, mask=None, relu=False, out_bf16=False):
    torch, ising = env
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.bfloat16 if out_bf16 else torch.float32, device="cuda")
    vp = ctypes.c_void_p
    rc = ising._lib.ising_tc_gemm(
        M, N, K, vp(A.data_ptr()), K, vp(B.data_ptr()), K,
        ctypes.cast(bias.data_ptr(), ctypes.POINTER(ctypes.c_float)) if bias is not None else None,
        vp(mask.data_ptr()) if mask is not None else None, N if mask is not None else 0, int(relu),
        vp(C.data_ptr()), N, int(out_bf16), vp(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, ising.ising_last_error()
    torch.cuda.synchronize()
    return C.float().cpu().numpy()


def _ref(A, B, bias=None, mask=None, relu=False):
    r = A.double().cpu().numpy() @ B.double().cpu().numpy().T
    if bias is not None:
        r += bias.double().cpu().numpy()[None, :]
    if relu:
        r = np.maximum(r, 0)
    if mask is not None:
        r = np.where(mask.float().cpu().numpy() > 0, r, 0)
    return r


@pytest.fixture(scope="module", autouse=True)
def _bind(env):
    torch, ising = env
    f = ising._lib.ising_tc_gemm
    f.argtypes = [ctypes.c_int32] * 3 + [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_int32, ctypes.POINTER(ctypes.c_float),
                                         ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_void_p]
    f.restype = ctypes.c_int32


@pytest.mark.parametrize("N", [32, 64, 128, 256])
@pytest.mark.parametrize("M,K", [(128, 64), (384, 256), (256, 4096)])
def test_plain_product(env, M, N, K):
    torch, _ = env
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N + K)
    A = torch.randn((M, K), generator=g).to(torch.bfloat16).cuda()
    B = torch.randn((N, K), generator=g).to(torch.bfloat16).cuda()
    got = _gemm(env, A, B)
    ref = _ref(A, B)
    scale = np.sqrt(K)
    assert np.abs(got - ref).max() <= 1e-4 * scale * 8, np.abs(got - ref).max()


def test_fused_epilogue_bias_relu_mask_bf16(env):
    torch, _ = env
    g = torch.Generator(device="cpu").manual_seed(5)
    M, N, K = 256, 256, 256
    A = torch.randn((M, K), generator=g).to(torch.bfloat16).cuda()
    B = (torch.randn((N, K), generator=g) * 0.1).to(torch.bfloat16).cuda()
    bias = torch.randn(N, generator=g).float().cuda()
    mask = torch.randn((M, N), generator=g).to(torch.bfloat16).cuda()
    got = _gemm(env, A, B, bias=bias, mask=mask, relu=True, out_bf16=True)
    ref = _ref(A, B, bias=bias, mask=mask, relu=True)
    assert np.abs(got - ref).max() <= 2e-2 * max(1.0, np.abs(ref).max() / 8)
    assert ((got == 0) == (ref == 0)).mean() > 0.999


def test_rejects_bad_shapes(env):
    torch, ising = env
    A = torch.zeros((100, 64), dtype=torch.bfloat16, device="cuda")
    B = torch.zeros((32, 64), dtype=torch.bfloat16, device="cuda")
    C = torch.zeros((100, 32), dtype=torch.float32, device="cuda")
    vp = ctypes.c_void_p
    rc = ising._lib.ising_tc_gemm(100, 32, 64, vp(A.data_ptr()), 64, vp(B.data_ptr()), 64, None,
                                  None, 0, 0, vp(C.data_ptr()), 32, 0, None)
    assert rc == -1
