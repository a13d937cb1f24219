"""Parity of the derived problems and triangular building blocks with the oracle.

TRSM/TRMM in all eight variants, TRTRI, TRULM (Sec. 3.2, Algorithms 2-4),
the in-place inverse and the reduced column echelon form (Algorithms 7-8),
rank profile and linear solving, each compared element by element with the
CPU oracle (or with its inverse/product, which the oracle pins) on seeded inputs.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1112_5717_gb300 import inputs
from tests._helpers import exact_matmul_mod, low_rank

pytestmark = pytest.mark.gpu

LEFT, UPPER, UNIT = 1, 2, 4


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint32).astype(np.int64)


def _tri(T, flags):
    """The triangle T denotes under `flags` (unit diagonal if UNIT)."""
    n = T.shape[0]
    E = np.triu(T, 1) if flags & UPPER else np.tril(T, -1)
    d = np.ones(n, dtype=np.int64) if flags & UNIT else np.diag(T).astype(np.int64)
    return E + np.diag(d)


@pytest.fixture(scope="module", params=[0, 1], ids=["plain", "tensor"])
def handle(request, cuda_lib):
    h = cuda_lib.Handle(engine=request.param, tc_min_k=1)
    yield h
    h.close()


@pytest.mark.parametrize("flags", range(8))
@pytest.mark.parametrize("n,other,p", [(1, 3, 7), (37, 50, 65521), (64, 64, 2), (65, 20, 251),
                                       (200, 90, 2147483647), (130, 129, 8388593)])
def test_trsm_trmm_variants(handle, flags, n, other, p):
    rng = np.random.default_rng(flags * 1000 + n + p % 1000)
    T = rng.integers(0, p, size=(n, n))
    T[np.arange(n), np.arange(n)] = rng.integers(1, p, size=n)   # invertible diagonal
    Te = _tri(T, flags)
    shape = (n, other) if flags & LEFT else (other, n)
    B = rng.integers(0, p, size=shape)
    Ti = oracle.inverse(Te, p).astype(np.int64)
    want_s = exact_matmul_mod(Ti, B, p) if flags & LEFT else exact_matmul_mod(B, Ti, p)
    want_m = exact_matmul_mod(Te, B, p) if flags & LEFT else exact_matmul_mod(B, Te, p)
    dT = _dev(T)
    dB = _dev(B)
    handle.trsm(flags, dT, dB, p)
    assert np.array_equal(_host(dB), want_s)
    dB = _dev(B)
    handle.trmm(flags, dT, dB, p)
    assert np.array_equal(_host(dB), want_m)
    assert np.array_equal(_host(dT), T)          # T is only read


@pytest.mark.parametrize("flags", [UPPER, UPPER | UNIT, 0, UNIT])
@pytest.mark.parametrize("n,p", [(1, 5), (64, 65521), (65, 251), (190, 1073741789), (128, 2)])
def test_trtri(handle, flags, n, p):
    rng = np.random.default_rng(n * 7 + flags)
    T = rng.integers(0, p, size=(n, n))
    T[np.arange(n), np.arange(n)] = rng.integers(1, p, size=n)
    Ti = oracle.inverse(_tri(T, flags), p).astype(np.int64)
    want = T.copy()
    mask = np.triu(np.ones((n, n), bool), 1) if flags & UPPER else np.tril(np.ones((n, n), bool), -1)
    if not flags & UNIT:
        mask |= np.eye(n, dtype=bool)
    want[mask] = Ti[mask]
    dT = _dev(T)
    handle.trtri(flags, dT, p)
    assert np.array_equal(_host(dT), want)


@pytest.mark.parametrize("n,p", [(1, 7), (40, 65521), (64, 3), (97, 8388593), (260, 2147483647)])
def test_trulm(handle, n, p):
    rng = np.random.default_rng(n)
    A = rng.integers(0, p, size=(n, n))
    U = np.triu(A, 1) + np.eye(n, dtype=np.int64)
    L = np.tril(A)
    want = exact_matmul_mod(U, L, p)
    dA = _dev(A)
    handle.trulm(dA, p)
    assert np.array_equal(_host(dA), want)


@pytest.mark.parametrize("n,p", [(1, 3), (50, 65521), (130, 8388593), (300, 2147483647), (257, 251),
                                 (96, 2)])
def test_inverse(handle, n, p):
    rng = np.random.default_rng(n + p % 97)
    for _ in range(10):
        A = rng.integers(0, p, size=(n, n))
        want = oracle.inverse(A, p)
        if want is not None:
            break
    assert want is not None
    dA = _dev(A)
    assert handle.inverse(dA, p)
    assert np.array_equal(_host(dA), want.astype(np.int64))


def test_inverse_singular_leaves_factors(handle):
    p = 65521
    rng = np.random.default_rng(1)
    A = low_rank(rng, 90, 90, 60, p)
    dA = _dev(A)
    assert not handle.inverse(dA, p)
    assert np.array_equal(_host(dA), oracle.cup_packed(A, p)["packed"].astype(np.int64))


RREF_CASES = [(7, 5, 3, 13), (60, 40, 40, 65521), (40, 60, 25, 251), (300, 130, 70, 8388593),
              (150, 150, 150, 2147483647), (200, 90, 0, 7), (256, 256, 100, 2), (129, 200, 128, 3)]


@pytest.mark.parametrize("m,n,r,p", RREF_CASES)
def test_rref(handle, m, n, r, p):
    rng = np.random.default_rng(m * n + r)
    A = low_rank(rng, m, n, r, p) if r < min(m, n) else rng.integers(0, p, size=(m, n))
    if r == 0:
        A = np.zeros((m, n), dtype=np.int64)
    want = oracle.rref(A, p, want_x=True)
    dA = _dev(A)
    rank, prof, X = handle.rref(dA, p, want_x=True)
    assert rank == want["rank"]
    assert np.array_equal(prof.cpu().numpy(), want["profile"])
    assert np.array_equal(_host(dA), want["R"].astype(np.int64))
    assert np.array_equal(_host(X), want["X"].astype(np.int64))


def test_rref_rank_deficient_workload(handle):
    p = inputs.P_23
    A = inputs.rank_deficient(m=700, n=256, r=150, p=p)
    want = oracle.rref(A, p)
    dA = _dev(A)
    rank, prof, _ = handle.rref(dA, p)
    assert rank == want["rank"] == 150
    assert np.array_equal(prof.cpu().numpy(), want["profile"])
    assert np.array_equal(_host(dA), want["R"].astype(np.int64))


@pytest.mark.parametrize("m,n,r,k,p", [(8, 6, 6, 1, 7), (90, 120, 50, 3, 65521), (150, 150, 150, 2, 251),
                                       (300, 200, 120, 5, 2147483647), (64, 64, 32, 4, 2)])
def test_solve(handle, m, n, r, k, p):
    rng = np.random.default_rng(m + n + r + k)
    A = low_rank(rng, m, n, r, p) if r < min(m, n) else rng.integers(0, p, size=(m, n))
    Y = rng.integers(0, p, size=(n, k))
    B = exact_matmul_mod(A, Y, p)
    s_o, X_o, r_o = oracle.solve(A, B, p)
    assert s_o == 0
    st, X, rank = handle.solve(_dev(A), _dev(B), p)
    assert st == 0 and rank == r_o
    assert np.array_equal(_host(X), X_o.astype(np.int64))
    if r < m:
        # a right-hand side outside the column space
        for i in range(m):
            e = np.zeros((m, 1), dtype=np.int64)
            e[i, 0] = 1
            if oracle.solve(A, e, p)[0] == 2:
                st2, _, _ = handle.solve(_dev(A), _dev(e), p)
                assert st2 == 2
                break


@pytest.mark.parametrize("m,n,p", [(600, 256, inputs.P_23), (100, 300, 65521), (64, 64, 2)])
def test_rank_profile(handle, m, n, p):
    A = inputs.rank_deficient(m=m, n=n, r=min(m, n) // 2, p=p) if p > 2 else inputs.dense_full(m=m, n=n, p=2)
    want = oracle.cup(A, p)
    r, prof = handle.rank_profile(_dev(A), p)
    assert r == want["rank"]
    assert np.array_equal(prof.cpu().numpy(), want["profile"])


@pytest.mark.parametrize("m,n,r,p", [(40, 60, 25, 65521), (64, 64, 64, 8388593), (100, 37, 20, 251),
                                     (30, 90, 0, 7), (130, 200, 120, 2147483647), (1, 5, 1, 2)])
def test_nullspace(handle, m, n, r, p):
    """cup_nullspace equals the oracle's basis (the last n - r columns of the echelon
    transform) bit for bit, and the basis is annihilated by A."""
    rng = np.random.default_rng(3 * m + n + r)
    A = np.zeros((m, n), dtype=np.int64) if r == 0 else (
        low_rank(rng, m, n, r, p) if r < min(m, n) else rng.integers(0, p, size=(m, n)))
    want = oracle.nullspace(A, p)
    rank, N = handle.nullspace(_dev(A), p)
    assert rank == want["rank"] == r
    got = _host(N.contiguous())
    assert got.shape == (n, n - r)
    assert np.array_equal(got, want["N"].astype(np.int64))
    if n - r:
        assert not exact_matmul_mod(A, got, p).any()


@pytest.mark.parametrize("m,n,r,p", [(50, 70, 30, 65521), (70, 50, 50, 8388593), (129, 200, 129, 251),
                                     (300, 100, 60, 2147483647), (64, 64, 0, 7), (1, 9, 1, 2)])
def test_ple(handle, m, n, r, p):
    """cup_ple equals the oracle's PLE bit for bit: [L\\E], the column rank profile and
    the row exchanges."""
    rng = np.random.default_rng(5 * m + n + r)
    A = np.zeros((m, n), dtype=np.int64) if r == 0 else (
        low_rank(rng, m, n, r, p) if r < min(m, n) else rng.integers(0, p, size=(m, n)))
    want = oracle.ple(A, p)
    dA = _dev(A)
    rank, prof, ipiv = handle.ple(dA, p)
    assert rank == want["rank"] == r
    assert np.array_equal(prof.cpu().numpy(), want["profile"])
    assert np.array_equal(ipiv.cpu().numpy(), want["ipiv"])
    assert np.array_equal(_host(dA), want["packed"].astype(np.int64))


@pytest.mark.parametrize("n,p", [(1, 7), (40, 65521), (64, 3), (97, 8388593), (260, 2147483647)])
def test_trlum(handle, n, p):
    """Algorithm 5: [L\\U] <- L U, checked against the product of the split factors."""
    rng = np.random.default_rng(n + 7)
    A = rng.integers(0, p, size=(n, n))
    want = oracle.trlum(A, p, unit_lower=True)
    dA = _dev(A)
    handle.trlum(dA, p)
    assert np.array_equal(_host(dA), want)


@pytest.mark.parametrize("m,n,p,rank", [(1, 1, 7, 1), (40, 13, 65521, 40), (64, 64, 3, 64),
                                        (97, 150, 8388593, 97), (130, 70, 2147483647, 130),
                                        (200, 33, 65521, 117), (129, 65, 2, 50), (70, 20, 251, 0)])
def test_inplace_mm(handle, m, n, p, rank):
    """Algorithm 9: B <- A B through CUP, two TRMMs and TRLUM; A comes back unchanged."""
    rng = np.random.default_rng(m * 31 + n + rank)
    if rank == m:
        A = rng.integers(0, p, size=(m, m))
    else:
        A = exact_matmul_mod(rng.integers(0, p, size=(m, rank)), rng.integers(0, p, size=(rank, m)), p)
    B = rng.integers(0, p, size=(m, n))
    want = oracle.inplace_mm(A, B, p)
    dA = _dev(A)
    dB = _dev(B)
    r = handle.inplace_mm(dA, dB, p)
    assert np.array_equal(_host(dB), want)
    assert np.array_equal(_host(dA), A % p)
    assert r == oracle.cup(A % p, p)["rank"]
