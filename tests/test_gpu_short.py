"""The one-launch short-K tensor update (mma.sync on digits made in shared memory):
bit-exact against the oracle for every limb count it serves (p below 2^8, 2^16,
2^24), inner dimensions around the 16-wide MMA step and the 64 / 128 / 256 variants,
ragged 64 x 64 tiles, extreme centred digits, the limits that send an update to
the tcgen05 launch instead, and the CUP factorisation with the path on and off."""
import numpy as np
import pytest

import oracle
from paper_1112_5717_gb300 import inputs

pytestmark = pytest.mark.gpu

PRIMES = [2, 3, 251, 257, 65521, 65537, 8388593, 16777213]


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.fixture(scope="module")
def short_handle(cuda_lib):
    h = cuda_lib.Handle(engine=cuda_lib.ENGINE_TENSOR, tc_min_k=1, short_k=256)
    yield h
    h.close()


@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (64, 64, 64), (65, 63, 15), (130, 77, 16), (7, 300, 17),
                                   (200, 129, 63), (64, 256, 65), (129, 64, 100), (3, 5, 127), (128, 130, 128),
                                   (65, 70, 129), (130, 64, 200), (64, 129, 255), (128, 128, 256)])
def test_short_mm_sub(cuda_lib, short_handle, p, M, N, K):
    rng = np.random.default_rng((M * 131 + N * 17 + K) ^ (p & 0xFFFF))
    A = rng.integers(0, p, size=(M, K))
    B = rng.integers(0, p, size=(K, N))
    C = rng.integers(0, p, size=(M, N))
    want = oracle.mm_sub(C, A, B, p)
    dC = _dev(C)
    short_handle.reset_stats()
    short_handle.mm_sub(dC, _dev(A), _dev(B), p, engine=cuda_lib.ENGINE_TENSOR)
    assert np.array_equal(_host(dC), want)
    assert short_handle.stats()["sk_launches"] == 1


@pytest.mark.parametrize("p", [251, 65521, 16777213])
@pytest.mark.parametrize("K", [64, 128, 256])
def test_short_mm_sub_extreme_digits(cuda_lib, short_handle, p, K):
    """(p - 1) / 2 and (p + 1) / 2 are the centred residues of largest magnitude, of both
    signs; with equal signs along K the fp32 partial sums reach their bound."""
    M, N = 96, 80
    rng = np.random.default_rng(p + K)
    lo, hi = (p - 1) // 2, (p + 1) // 2
    A = np.where(rng.random((M, K)) < 0.5, lo, hi)
    B = np.where(rng.random((K, N)) < 0.5, lo, hi)
    A[: M // 2] = hi
    B[:, : N // 2] = hi
    C = rng.integers(0, p, size=(M, N))
    want = oracle.mm_sub(C, A, B, p)
    dC = _dev(C)
    short_handle.mm_sub(dC, _dev(A), _dev(B), p, engine=cuda_lib.ENGINE_TENSOR)
    assert np.array_equal(_host(dC), want)


def test_short_path_limits(cuda_lib, short_handle):
    """K above 256, p above 2^24 and more than 2^21 outputs go to the tcgen05 launch."""
    p = 65521
    rng = np.random.default_rng(5)
    for (M, N, K, q) in [(64, 64, 257, p), (64, 64, 64, 16777259), (2048, 1025, 32, p)]:
        A = rng.integers(0, q, size=(M, K))
        B = rng.integers(0, q, size=(K, N))
        C = rng.integers(0, q, size=(M, N))
        want = oracle.mm_sub(C, A, B, q)
        dC = _dev(C)
        short_handle.reset_stats()
        short_handle.mm_sub(dC, _dev(A), _dev(B), q, engine=cuda_lib.ENGINE_TENSOR)
        st = short_handle.stats()
        assert st["sk_launches"] == 0 and st["tc_launches"] == 1, (M, N, K, q)
        assert np.array_equal(_host(dC), want)


@pytest.mark.parametrize("short_k", [0, 64, 128, 256])
@pytest.mark.parametrize("name,p", [("dense", 65521), ("dense", 251), ("rank_def", 8388593)])
def test_factor_with_short_updates(cuda_lib, short_k, name, p):
    if name == "dense":
        A = inputs.dense_full(n=448, p=p)
    else:
        A = inputs.rank_deficient(m=640, n=300, r=170, p=p)
    d = oracle.cup_packed(A, p)
    h = cuda_lib.Handle(engine=cuda_lib.ENGINE_TENSOR, tc_min_k=1, short_k=short_k)
    dA = _dev(A)
    h.reset_stats()
    r, prof, ipiv = h.factor(dA, p)
    assert r == d["rank"]
    assert np.array_equal(prof[:r].cpu().numpy(), d["profile"])
    assert np.array_equal(_host(dA), d["packed"])
    st = h.stats()
    assert (st["sk_launches"] > 0) == (short_k > 0)
    h.close()
