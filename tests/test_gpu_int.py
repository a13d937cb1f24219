"""Integer determinant and rank by multi-modular reduction (Sec. 1: problems over
Z reduced to prime fields), against the oracle's exact integer elimination
(small sizes) and closed forms that hold at any size.

Both sides of the path are covered: images with min(m, n) <= 512 go through the
batched launch, larger ones through one full-device CUP per prime.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _dev64(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.int64))).cuda()


@pytest.fixture(scope="module", params=[0, 1], ids=["plain", "tensor"])
def handle(request, cuda_lib):
    h = cuda_lib.Handle(engine=request.param)
    yield h
    h.close()


def _ldu(rng, n, span=2, dmax=5):
    """A = L D U with unit triangular L, U (entries in [-span, span]) and a nonzero
    diagonal D: det A = prod D exactly; returns (A as int64, det)."""
    L = np.tril(rng.integers(-span, span + 1, size=(n, n)), -1) + np.eye(n, dtype=np.int64)
    U = np.triu(rng.integers(-span, span + 1, size=(n, n)), 1) + np.eye(n, dtype=np.int64)
    d = rng.integers(1, dmax + 1, size=n) * rng.choice([-1, 1], size=n)
    A = (L.astype(object) * d.astype(object)).dot(U.astype(object))
    det = 1
    for x in d:
        det *= int(x)
    return np.array(A, dtype=np.int64), det


@pytest.mark.parametrize("n,bits", [(1, 20), (2, 62), (5, 40), (33, 20), (64, 8), (130, 12)])
def test_int_det_matches_oracle(handle, n, bits):
    rng = np.random.default_rng(n * 7 + bits)
    A = rng.integers(-(1 << bits), 1 << bits, size=(n, n), dtype=np.int64)
    det, rank, cert, k = handle.int_det(_dev64(A))
    assert cert and k >= 1
    assert det == oracle.int_det(A)
    assert rank == (n if det != 0 else oracle.int_rank(A))


def test_int_det_extreme_entries(handle):
    """INT64_MIN and INT64_MAX entries reduce correctly (signed residues)."""
    lo, hi = np.iinfo(np.int64).min, np.iinfo(np.int64).max
    A = np.array([[lo, hi, 3], [hi, 5, lo], [-7, lo, hi]], dtype=np.int64)
    det, rank, cert, _ = handle.int_det(_dev64(A))
    assert cert and det == oracle.int_det(A) and rank == 3


@pytest.mark.parametrize("n", [200, 513, 600])
def test_int_det_closed_form(handle, n):
    """det(L D U) = prod D at sizes on both sides of the batched limit."""
    rng = np.random.default_rng(n)
    A, want = _ldu(rng, n)
    det, rank, cert, k = handle.int_det(_dev64(A))
    assert cert and det == want and rank == n
    assert k >= 2


def test_int_det_singular_and_degenerate(handle):
    rng = np.random.default_rng(4)
    A = rng.integers(-100, 100, size=(40, 40))
    A[17] = 3 * A[2] - A[30]                 # dependent row
    det, rank, cert, _ = handle.int_det(_dev64(A))
    assert det == 0 and cert and rank == oracle.int_rank(A) == 39
    Z = np.zeros((9, 9), dtype=np.int64)
    assert handle.int_det(_dev64(Z))[:3] == (0, 0, True)
    I = np.eye(70, dtype=np.int64)
    assert handle.int_det(_dev64(I))[:3] == (1, 70, True)
    P = np.eye(6, dtype=np.int64)[[1, 0, 2, 3, 4, 5]]
    assert handle.int_det(_dev64(-P))[0] == -1           # (-1)^6 det P, P one transposition
    import torch
    assert handle.int_det(torch.zeros((0, 0), dtype=torch.int64, device="cuda"))[:3] == (1, 0, True)


def test_int_det_with_given_primes(handle):
    """With too few primes the result is det modulo their product (symmetric
    range) and is flagged uncertified; with enough it is exact."""
    import paper_1112_5717_gb300 as cup
    rng = np.random.default_rng(11)
    A = rng.integers(-(1 << 30), 1 << 30, size=(24, 24))
    want = oracle.int_det(A)
    primes = cup.primes_below(1 << 30, 3)
    M = primes[0] * primes[1] * primes[2]
    det, _, cert, k = handle.int_det(_dev64(A), primes)
    assert not cert and k == 3
    sym = want % M
    if sym > M // 2:
        sym -= M
    assert det == sym
    many = cup.primes_below(1 << 31, 40)
    det, _, cert, k = handle.int_det(_dev64(A), many)
    assert cert and k == 40 and det == want


@pytest.mark.parametrize("m,n,r", [(40, 30, 17), (1, 9, 1), (50, 50, 50), (64, 20, 0)])
def test_int_rank_matches_oracle(handle, m, n, r):
    rng = np.random.default_rng(m + n + r)
    X = rng.integers(-5, 6, size=(m, r)).astype(object)
    Y = rng.integers(-5, 6, size=(r, n)).astype(object)
    A = np.array(X.dot(Y), dtype=np.int64) if r else np.zeros((m, n), dtype=np.int64)
    rank, cert, k = handle.int_rank(_dev64(A))
    assert cert and rank == oracle.int_rank(A)


@pytest.mark.parametrize("m,n,r", [(700, 650, 300), (520, 900, 519)])
def test_int_rank_large(handle, m, n, r):
    """Large ranks on the per-prime path: the factors' construction bounds the
    rank by r, and the oracle's CUP modulo one prime shows it reaches r."""
    rng = np.random.default_rng(m * n + r)
    X = rng.integers(-3, 4, size=(m, r)).astype(object)
    Y = rng.integers(-3, 4, size=(r, n)).astype(object)
    A = np.array(X.dot(Y), dtype=np.int64)
    q = 1073741789
    assert oracle.cup((A % q).astype(np.uint32), q)["rank"] == r
    rank, cert, k = handle.int_rank(_dev64(A))
    assert cert and rank == r


@pytest.mark.parametrize("path", [1, 2])
def test_int_paths_agree(cuda_lib, path):
    """The batched launch and the per-prime factorisations give the same results."""
    h = cuda_lib.Handle(int_path=path)
    rng = np.random.default_rng(path)
    A, want = _ldu(rng, 150)
    det, rank, cert, _ = h.int_det(_dev64(A))
    assert cert and det == want and rank == 150
    X = rng.integers(-4, 5, size=(90, 40))
    Y = rng.integers(-4, 5, size=(40, 120))
    B = X @ Y
    assert h.int_rank(_dev64(B))[:2] == (oracle.int_rank(B), True)
    h.close()
