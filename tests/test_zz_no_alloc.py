"""The allocation-free Schur update against the handle-based one and the oracle.

cup_mm_sub_noalloc serves callers that cannot call cudaMalloc: a process whose
device memory is all reserved by its own fixed-size pool, or code that must not
allocate after start-up because cudaMalloc and cudaFree may synchronise the whole
device. Its limb scratch is a fixed array inside the library. This test calls it
twice in a row through the C ABI and requires both results to equal, bit for bit,
those of cup_mm_sub on the tensor engine for the same inputs and the oracle's
C - A B mod p (Algorithm 1 with alpha = -1, beta = 1); it also checks that a product
too large for the scratch is refused without touching C. The file is named so that
pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _call_noalloc(lib, C, A, B, p):
    import torch
    M, N = C.shape
    K = A.shape[1]
    st = lib.cup_mm_sub_noalloc(C.data_ptr(), C.stride(0), A.data_ptr(), A.stride(0), B.data_ptr(),
                                B.stride(0), M, N, K, p,
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


@pytest.mark.parametrize("p", [251, 65521, 8388593, 2147483647])
def test_noalloc_equals_handle_path_twice(cuda_lib, p):
    import torch
    lib = cuda_lib.load()
    h = cuda_lib.Handle(engine=cuda_lib.ENGINE_TENSOR, tc_min_k=1)
    rng = np.random.default_rng(p & 0xFFFF)
    for call, (M, N, K) in enumerate([(300, 260, 700), (129, 77, 1030)]):
        A = rng.integers(0, p, size=(M, K))
        B = rng.integers(0, p, size=(K, N))
        C = rng.integers(0, p, size=(M, N))
        want = _dev(C)
        h.mm_sub(want, _dev(A), _dev(B), p, engine=cuda_lib.ENGINE_TENSOR)
        got = _dev(C)
        assert _call_noalloc(lib, got, _dev(A), _dev(B), p) == 0, f"call {call}"
        torch.cuda.synchronize()
        assert torch.equal(got, want), f"call {call} differs from cup_mm_sub"
        ref = oracle.mm_sub(C, A, B, p)
        assert np.array_equal(got.cpu().numpy().view(np.uint32), ref), f"call {call} differs from the oracle"
    h.close()


def test_noalloc_rejects_products_beyond_its_scratch(cuda_lib):
    import torch
    lib = cuda_lib.load()
    p = 2147483647                      # 4 limbs: 4 * (M + N) * K * 2 bytes
    M = N = 2048
    K = 1024                            # 32 MiB of limb planes > 16 MiB
    A = torch.zeros((M, K), dtype=torch.int32, device="cuda")
    B = torch.zeros((K, N), dtype=torch.int32, device="cuda")
    C = torch.ones((M, N), dtype=torch.int32, device="cuda")
    assert _call_noalloc(lib, C, A, B, p) == -8
    torch.cuda.synchronize()
    assert int(C.sum().item()) == M * N
