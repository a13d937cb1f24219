"""Exactness of the tcgen05 limb Schur update C <- C - A B mod p.

The tensor engine carries 8-bit centred digits in bf16 and accumulates in
fp32; these tests compare it bit for bit with the oracle across every limb
count (p below 2^8, 2^16, 2^24, 2^31), ragged tile edges, inner dimensions
that cross the exact-accumulation chunk boundary, and extreme digits.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

PRIMES = [2, 3, 251, 257, 65521, 65537, 8388593, 16777213, 1073741789, 2147483647]


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint32)


def _limbs(p):
    return 1 if p < 2 ** 8 else 2 if p < 2 ** 16 else 3 if p < 2 ** 24 else 4


def _chunk(p):
    return (1024 // _limbs(p)) // 64 * 64


@pytest.fixture(scope="module")
def tensor_handle(cuda_lib):
    h = cuda_lib.Handle(engine=cuda_lib.ENGINE_TENSOR, tc_min_k=1)
    yield h
    h.close()


@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (128, 128, 64), (130, 77, 45), (200, 333, 600),
                                   (257, 130, 1100), (64, 300, 2049), (300, 700, 4100)])
def test_tensor_mm_sub_random(cuda_lib, tensor_handle, p, M, N, K):
    rng = np.random.default_rng((M * 31 + N * 7 + K) ^ (p & 0xFFFF))
    A = rng.integers(0, p, size=(M, K))
    B = rng.integers(0, p, size=(K, N))
    C = rng.integers(0, p, size=(M, N))
    want = oracle.mm_sub(C, A, B, p)
    dC = _dev(C)
    tensor_handle.mm_sub(dC, _dev(A), _dev(B), p, engine=cuda_lib.ENGINE_TENSOR)
    assert np.array_equal(_host(dC), want)


@pytest.mark.parametrize("p", PRIMES[2:])
def test_tensor_mm_sub_extreme_digits(cuda_lib, tensor_handle, p):
    """Entries (p-1)/2 and (p+1)/2 give the largest centred digits of both signs;
    K is a whole number of exact-accumulation chunks plus one, so every fp32
    accumulator reaches its bound."""
    K = 2 * _chunk(p) + 1
    M, N = 160, 192
    rng = np.random.default_rng(p & 0xFFFF)
    lo, hi = (p - 1) // 2, (p + 1) // 2
    A = np.where(rng.random((M, K)) < 0.5, lo, hi)
    B = np.where(rng.random((K, N)) < 0.5, lo, hi)
    A[:, ::3] = lo
    B[::3, :] = lo          # runs of equal sign push the partial sums to the bound
    C = rng.integers(0, p, size=(M, N))
    want = oracle.mm_sub(C, A, B, p)
    dC = _dev(C)
    tensor_handle.mm_sub(dC, _dev(A), _dev(B), p, engine=cuda_lib.ENGINE_TENSOR)
    assert np.array_equal(_host(dC), want)


def test_tensor_mm_sub_strided_views(cuda_lib, tensor_handle):
    """Operands as views into one matrix with a leading dimension, as the CUP
    recursion passes them (G, V1 and H are blocks of A)."""
    import torch
    p = 65521
    rng = np.random.default_rng(5)
    big = rng.integers(0, p, size=(700, 900)).astype(np.uint32)
    dbig = _dev(big)
    r0, c0, M, N, K = 300, 250, 400, 650, 250
    Cv = dbig[r0:r0 + M, c0:c0 + N]
    Av = dbig[r0:r0 + M, c0 - K:c0]
    Bv = dbig[0:K, c0:c0 + N]
    want = oracle.mm_sub(big[r0:r0 + M, c0:c0 + N], big[r0:r0 + M, c0 - K:c0], big[0:K, c0:c0 + N], p)
    tensor_handle.mm_sub(Cv, Av, Bv, p, engine=cuda_lib.ENGINE_TENSOR)
    torch.cuda.synchronize()
    out = _host(dbig)
    assert np.array_equal(out[r0:r0 + M, c0:c0 + N], want)
    mask = np.ones(big.shape, dtype=bool)
    mask[r0:r0 + M, c0:c0 + N] = False
    assert np.array_equal(out[mask], big[mask])
