"""The surrogate's tcgen05 BF16 GEMM (synax_gemm_bf16) against a plain
PyTorch FP32 matmul of the same BF16 inputs: C = A B^T, FP32 accumulation."""
import ctypes

import numpy as np
import pytest

from paper_2410_01136_gb300 import _native

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2410_01136_gb300 import build
    build()
    return _t


def run_gemm(torch, A, B, ldc=None):
    M, K = A.shape
    N = B.shape[0]
    ldc = ldc or N
    C = torch.full((M, ldc), float("nan"), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = _native.lib().synax_gemm_bf16(ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.c_void_p(B.data_ptr()),
                                       B.stride(0), M, N, K, ctypes.c_void_p(C.data_ptr()), ldc,
                                       ctypes.c_void_p(err.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, rc
    torch.cuda.synchronize()
    assert int(err.item()) == 0, "bounded wait expired"
    return C[:, :N]


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (128, 64, 64), (256, 1024, 1024), (200, 9216, 1024),
                                   (1024, 64, 512), (512, 300, 128), (77, 256, 192), (1, 1024, 64),
                                   (12345, 1100, 64)])          # two waves of 256-column tiles, ragged edges
def test_gemm_matches_fp32_matmul(torch, M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M * 7919 + N * 31 + K)
    A = torch.randn((M, K), generator=g, device="cuda").to(torch.bfloat16)
    B = torch.randn((N, K), generator=g, device="cuda").to(torch.bfloat16)
    C = run_gemm(torch, A, B)
    ref = A.float() @ B.float().T
    err = (C - ref).abs().max().item()
    assert err <= 1e-4 * ref.abs().max().item() + 1e-5, err


def test_gemm_unaligned_output_pitch(torch):
    """An output pitch that is not a multiple of 4 floats takes the direct-store epilogue."""
    A = torch.randn((200, 128), device="cuda").to(torch.bfloat16)
    B = torch.randn((300, 128), device="cuda").to(torch.bfloat16)
    C = run_gemm(torch, A, B, ldc=301)
    ref = A.float() @ B.float().T
    assert (C - ref).abs().max().item() <= 1e-4 * ref.abs().max().item()


def test_gemm_row_pitch_and_validation(torch):
    A = torch.randn((130, 128), device="cuda").to(torch.bfloat16)[:, :64]     # pitch 128, K 64
    B = torch.randn((96, 64), device="cuda").to(torch.bfloat16)
    C = run_gemm(torch, A, B, ldc=100)
    ref = A.float() @ B.float().T
    assert (C - ref).abs().max().item() <= 1e-4 * ref.abs().max().item()
    L = _native.lib()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    Cbad = torch.empty((4, 4), device="cuda")
    # K not a multiple of 64
    assert L.synax_gemm_bf16(ctypes.c_void_p(A.data_ptr()), 128, ctypes.c_void_p(B.data_ptr()), 64, 4, 4, 32,
                             ctypes.c_void_p(Cbad.data_ptr()), 4, ctypes.c_void_p(err.data_ptr()), None) \
        == _native.SYNAX_EINVAL


def test_bounded_wait_gives_up_and_context_survives(torch):
    """A wait on an mbarrier that nothing arrives at ends by its clock limit
    with the error word set, its CTA frees its TMEM, and the context stays
    usable: a GEMM (which allocates TMEM on every SM it runs on) still runs
    and matches afterwards."""
    import time
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    cycles = torch.zeros(1, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc = _native.lib().synax_wait_selftest(ctypes.c_void_p(err.data_ptr()), ctypes.c_void_p(cycles.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, rc
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    assert int(err.item()) == 1
    assert int(cycles.item()) > 2_000_000_000          # the limit, in SM clocks
    assert 0.3 < elapsed < 30.0, elapsed                # ~1 s at 2 GHz
    A = torch.randn((256, 512), device="cuda").to(torch.bfloat16)
    B = torch.randn((1024, 512), device="cuda").to(torch.bfloat16)
    C = run_gemm(torch, A, B)
    ref = A.float() @ B.float().T
    assert (C - ref).abs().max().item() <= 1e-4 * ref.abs().max().item()
