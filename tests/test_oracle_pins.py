"""Pins of the CPU oracle against definitions, closed forms and brute force.

These run on the CPU only. Each pins the oracle to something other than
itself, chosen so that a dropped term, a wrong sign, a wrong index or a
transposed operand in the oracle fails at least one of them:

* rank and row rank profile against the span definition (Sec. 2), exhaustively
  over all 3x3 matrices of GF(3) and all 4x4 matrices of GF(2);
* A P^T = C U, checked with exact integer products, plus the shapes the
  decomposition promises (C column echelon, U unit upper; Proposition 1);
* the pivot rule and the values of C and U against Schur-complement minors
  computed with the Leibniz formula (C, U are unique given P, Proposition 1);
* determinant against the Leibniz formula; inverse against A A^{-1} = I;
* reduced column echelon form against its uniqueness under A -> A G;
* the worked 7x5 example of Sec. 2.2 (row rank profile [0, 3, 4]);
* the operation count against 2mnr - (m+n)r^2 + 2/3 r^3 (Sec. 4.2).
"""
from __future__ import annotations

import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1112_5717_gb300 import inputs
from tests._helpers import (exact_matmul_mod, leibniz_det, low_rank, perm_matrix_from_ipiv,
                            random_invertible, span_profile)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _check_cup(A, p, d):
    A = np.asarray(A, dtype=np.int64)
    m, n = A.shape
    r = d["rank"]
    C = d["C"].astype(np.int64)
    U = d["U"].astype(np.int64)
    prof = list(d["profile"])
    ipiv = list(d["ipiv"])
    # A P^T = C U exactly (P^T as the product of the recorded transpositions)
    Pt = perm_matrix_from_ipiv(ipiv, n)
    lhs = exact_matmul_mod(A, Pt, p)
    rhs = exact_matmul_mod(C, U, p)
    assert np.array_equal(lhs, rhs)
    # C: column echelon, pivots on the profile rows, columns >= r zero
    assert prof == sorted(prof) and len(set(prof)) == r
    for t in range(r):
        assert C[prof[t], t] != 0
        assert not C[: prof[t], t].any()
    assert not C[:, r:].any()
    # U: unit upper triangular, rows >= r identity
    assert np.array_equal(np.diag(U), np.ones(n, dtype=np.int64))
    assert not np.tril(U, -1).any()
    assert np.array_equal(U[r:], np.eye(n, dtype=np.int64)[r:])
    # transpositions only move a column to a later position
    assert all(ipiv[t] >= t for t in range(r))


def test_modinv_against_fermat():
    for p in (2, 3, 5, 7, 251, 65521, 8388593, 1073741789, 2147483647):
        rng = np.random.default_rng(p)
        xs = range(1, p) if p < 300 else rng.integers(1, p, size=200)
        for a in xs:
            a = int(a)
            inv = oracle.modinv(a, p)
            assert inv == pow(a, p - 2, p)
            assert a * inv % p == 1
    assert oracle.modinv(0, 7) == 0


@pytest.mark.parametrize("p,n", [(3, 3), (2, 4)])
def test_rank_profile_exhaustive(p, n):
    """Every n x n matrix over GF(p): rank and profile equal the span definition
    and A P^T = C U holds exactly."""
    cache = {}
    count = 0
    for flat in itertools.product(range(p), repeat=n * n):
        A = np.array(flat, dtype=np.uint32).reshape(n, n)
        d = oracle.cup(A, p)
        prof = span_profile(A, p)
        assert d["rank"] == len(prof)
        assert list(d["profile"]) == prof
        # exact identity on a deterministic subsample (every matrix would be slow)
        if count % 37 == 0:
            _check_cup(A, p, d)
        count += 1
        cache[d["rank"]] = cache.get(d["rank"], 0) + 1
    assert sum(cache.values()) == p ** (n * n)
    # number of full-rank matrices: prod_{k<n} (p^n - p^k)
    full = 1
    for k in range(n):
        full *= p ** n - p ** k
    assert cache[n] == full


@pytest.mark.parametrize("shape,p,rank", [((6, 9), 7, 4), ((9, 5), 5, 3), ((8, 8), 65521, 8),
                                          ((12, 7), 2, 5), ((5, 5), 251, 0), ((1, 6), 13, 1),
                                          ((6, 1), 13, 1), ((40, 33), 8388593, 20)])
def test_cup_identity_and_shape(shape, p, rank):
    rng = np.random.default_rng(hash((shape, p, rank)) & 0xFFFF)
    m, n = shape
    A = low_rank(rng, m, n, rank, p) if rank < min(m, n) else rng.integers(0, p, size=(m, n))
    A[rng.integers(0, m)] = 0
    d = oracle.cup(A, p)
    _check_cup(A, p, d)
    assert list(d["profile"]) == span_profile(A, p) if p ** min(rank + 1, n) < 5000 else True


def _minor(A, rows, cols, p):
    return leibniz_det(np.asarray(A, dtype=np.int64)[np.ix_(rows, cols)], p)


@pytest.mark.parametrize("seed", range(12))
def test_pivot_rule_and_values_by_minors(seed):
    """Pivot choice, C and U from Schur complements (ratios of minors).

    The residual of row i at column c after eliminating pivots 0..t-1 is
    det(A[rows i_0..i_{t-1}, i; cols S_t, c]) / det(A[rows i_0..i_{t-1}; cols S_t])
    where S_t are the pivot columns in position order. So: the pivot of step
    t is the first position (in the order after transpositions 0..t-1) where
    that minor is nonzero; rows skipped between i_{t-1} and i_t have all such
    minors zero; C[i][t] and U[t][q] are the corresponding ratios."""
    rng = np.random.default_rng(1000 + seed)
    p = [5, 7, 11, 13][seed % 4]
    m, n = [(5, 5), (5, 4), (4, 6), (6, 5)][seed % 4]
    r = min(m, n) - seed % 3
    A = low_rank(rng, m, n, r, p)
    # force column swaps: zero a few leading columns of some rows
    A[0, : seed % 3] = 0
    d = oracle.cup(A, p)
    _check_cup(A, p, d)
    rank, prof, ipiv = d["rank"], list(d["profile"]), list(d["ipiv"])
    C, U = d["C"].astype(np.int64), d["U"].astype(np.int64)
    perm_final = oracle.perm_from_ipiv(ipiv, n)
    perm = np.arange(n)
    prev_row = -1
    for t in range(rank + 1):
        S = list(perm_final[:t])
        base = _minor(A, prof[:t], S, p) if t else 1
        assert base != 0
        inv_base = pow(base, p - 2, p)
        last = prof[t] if t < rank else m
        # rows strictly between profile rows: every residual is zero
        for i in range(prev_row + 1, last):
            for q in range(t, n):
                assert _minor(A, prof[:t] + [i], S + [int(perm[q])], p) == 0
        if t == rank:
            break
        i_t = prof[t]
        res = [(_minor(A, prof[:t] + [i_t], S + [int(perm[q])], p) * inv_base) % p for q in range(n)]
        first = next(q for q in range(t, n) if res[q] != 0)
        assert first == ipiv[t]
        perm[[t, first]] = perm[[first, t]]
        assert int(perm[t]) == int(perm_final[t])
        piv = res[first]
        # C column t: residual of each row at pivot t's column
        for i in range(m):
            if i < i_t:
                assert C[i, t] == 0
            else:
                val = _minor(A, prof[:t] + [i], S + [int(perm_final[t])], p) * inv_base % p
                assert C[i, t] == val
        # U row t in the final column order
        full = _minor(A, prof[: t + 1], list(perm_final[: t + 1]), p)
        assert full == piv * base % p
        inv_full = pow(full, p - 2, p)
        for q in range(t + 1, n):
            val = _minor(A, prof[: t + 1], list(perm_final[:t]) + [int(perm_final[q])], p) * inv_full % p
            assert U[t, q] == val
        prev_row = i_t


def test_pack_layout():
    p = 13
    rng = np.random.default_rng(5)
    A = low_rank(rng, 7, 5, 3, p)
    d = oracle.cup_packed(A, p)
    r, C, U, P = d["rank"], d["C"], d["U"], d["packed"]
    for i in range(7):
        for j in range(5):
            if i < r and j > i:
                assert P[i, j] == U[i, j]
            elif j < r and j <= i:
                assert P[i, j] == C[i, j]
            else:
                assert P[i, j] == 0


@pytest.mark.parametrize("n,p", [(1, 7), (2, 5), (3, 13), (4, 251), (5, 65521), (5, 2)])
def test_det_leibniz(n, p):
    rng = np.random.default_rng(n * 100 + p % 97)
    for trial in range(20):
        A = rng.integers(0, p, size=(n, n))
        if trial % 5 == 4 and n > 1:
            A[-1] = (2 * A[0]) % p       # singular
        assert oracle.det(A, p) == leibniz_det(A, p)


def test_det_multiplicative():
    p = 8388593
    rng = np.random.default_rng(3)
    X = rng.integers(0, p, size=(24, 24))
    Y = rng.integers(0, p, size=(24, 24))
    XY = exact_matmul_mod(X, Y, p)
    assert oracle.det(XY, p) == oracle.det(X, p) * oracle.det(Y, p) % p


@pytest.mark.parametrize("n,p", [(1, 3), (6, 7), (17, 65521), (30, 1073741789)])
def test_inverse(n, p):
    rng = np.random.default_rng(n)
    A = random_invertible(rng, n, p)
    perm = rng.permutation(n)
    A = A[perm]
    Ai = oracle.inverse(A, p)
    assert Ai is not None
    assert np.array_equal(exact_matmul_mod(A, Ai, p), np.eye(n, dtype=np.int64))
    assert np.array_equal(exact_matmul_mod(Ai, A, p), np.eye(n, dtype=np.int64))
    if n > 1:
        B = A.copy()
        B[1] = B[0]
        assert oracle.inverse(B, p) is None


@pytest.mark.parametrize("m,n,r,p", [(7, 5, 3, 13), (10, 10, 6, 65521), (6, 12, 6, 5), (15, 9, 9, 251)])
def test_rref_uniqueness(m, n, r, p):
    rng = np.random.default_rng(m * n + r)
    A = low_rank(rng, m, n, r, p)
    d = oracle.rref(A, p, want_x=True)
    R, X, rank, prof = d["R"].astype(np.int64), d["X"].astype(np.int64), d["rank"], list(d["profile"])
    assert rank == r
    assert prof == span_profile(A, p) if p ** r < 5000 else True
    # A X = R
    assert np.array_equal(exact_matmul_mod(A, X, p), R)
    # reduced column echelon shape
    assert not R[:, r:].any()
    for t in range(r):
        assert R[prof[t], t] == 1
        assert not R[: prof[t], t].any()
        row = R[prof[t]].copy()
        row[t] = 0
        assert not row.any()
    # invariance under right multiplication by an invertible matrix
    G = random_invertible(rng, n, p)
    d2 = oracle.rref(exact_matmul_mod(A, G, p), p)
    assert np.array_equal(d2["R"].astype(np.int64), R)
    # agreement with the CUP route: R = A P^T U D L, i.e. column space and profile
    c = oracle.cup(A, p)
    assert c["rank"] == rank and list(c["profile"]) == prof


@pytest.mark.parametrize("m,n,r,p", [(8, 6, 6, 7), (9, 12, 5, 65521), (6, 6, 6, 8388593)])
def test_solve(m, n, r, p):
    rng = np.random.default_rng(m + n + r)
    A = low_rank(rng, m, n, r, p)
    Y = rng.integers(0, p, size=(n, 3))
    B = exact_matmul_mod(A, Y, p)
    s, X, rank = oracle.solve(A, B, p)
    assert s == 0 and rank == r
    assert np.array_equal(exact_matmul_mod(A, X, p), B)
    # supported on the pivot columns only
    c = oracle.cup(A, p)
    perm = oracle.perm_from_ipiv(c["ipiv"], n)
    free = perm[rank:]
    assert not X[free].any()
    if r < m:
        # a right-hand side outside the column space is reported as inconsistent
        B2 = B.copy()
        w = np.zeros(m, dtype=np.int64)
        # find a vector not in the column space: the residual direction of a unit vector
        for i in range(m):
            e = np.zeros((m, 1), dtype=np.int64)
            e[i, 0] = 1
            s2, _, _ = oracle.solve(A, e, p)
            if s2 == 2:
                w = e[:, 0]
                break
        B2[:, 0] = (B2[:, 0] + w) % p
        s3, _, _ = oracle.solve(A, B2, p)
        assert s3 == 2


def test_mm_sub_exact():
    for (M, N, K, p) in [(5, 7, 3, 13), (33, 17, 65, 65521), (20, 20, 300, 2147483647), (4, 4, 0, 5)]:
        rng = np.random.default_rng(M * N + K)
        A = rng.integers(0, p, size=(M, K))
        B = rng.integers(0, p, size=(K, N))
        C = rng.integers(0, p, size=(M, N))
        got = oracle.mm_sub(C, A, B, p).astype(np.int64)
        want = (C.astype(object) - exact_matmul_mod(A, B, p).astype(object)) % p
        assert np.array_equal(got, want.astype(np.int64))


def test_trsm_variants():
    p = 65521
    rng = np.random.default_rng(9)
    n, m = 19, 11
    U = np.triu(rng.integers(0, p, size=(n, n)), 1) + np.eye(n, dtype=np.int64) * 12345  # diag ignored
    Uu = np.triu(U, 1) + np.eye(n, dtype=np.int64)
    B = rng.integers(0, p, size=(m, n))
    X = oracle.trsm_right_upper_unit(U, B, p).astype(np.int64)
    assert np.array_equal(exact_matmul_mod(X, Uu, p), B)
    B2 = rng.integers(0, p, size=(n, 4))
    X2 = oracle.trsm_left_upper_unit(U, B2, p).astype(np.int64)
    assert np.array_equal(exact_matmul_mod(Uu, X2, p), B2)
    L = np.tril(rng.integers(0, p, size=(n, n)), -1) + np.diag(rng.integers(1, p, size=n))
    X3 = oracle.trsm_left_lower_nonunit(L, B2, p).astype(np.int64)
    assert np.array_equal(exact_matmul_mod(L, X3, p), B2)


def test_laswp_matches_permutation_matrix():
    rng = np.random.default_rng(4)
    n = 9
    A = rng.integers(0, 100, size=(5, n))
    ipiv = [2, 1, 7, 3, 8]
    got = oracle.laswp_cols(A, ipiv).astype(np.int64)
    want = A @ perm_matrix_from_ipiv(ipiv, n)
    assert np.array_equal(got, want)


def test_golden_example_7x5():
    """Sec. 2.2's worked example: a 7x5 matrix whose row rank profile is
    [0, 3, 4]; C has its pivots at (0,0), (3,1), (4,2) (the barred entries of
    the example) and zeros above them."""
    path = os.path.join(GOLDEN, "example_7x5_profile_0_3_4.txt")
    p, A = None, []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("p="):
            p = int(line[2:])
            continue
        A.append([int(x) for x in line.split()])
    A = np.array(A, dtype=np.int64)
    assert A.shape == (7, 5)
    d = oracle.cup(A, p)
    assert d["rank"] == 3
    assert list(d["profile"]) == [0, 3, 4]
    C = d["C"]
    assert C[0, 0] and C[3, 1] and C[4, 2]
    assert not C[:3, 1].any() and not C[:4, 2].any() and not C[:, 3:].any()
    _check_cup(A, p, d)


def test_opcount_leading_term():
    """The plain elimination's count approaches 2mnr - (m+n)r^2 + 2/3 r^3 (Sec. 4.2)
    for a generic rank profile [0..r-1]: the difference is O(mn + r^2)."""
    for (m, n, r) in [(400, 400, 400), (800, 300, 300), (600, 900, 250)]:
        prof = np.arange(r)
        got = oracle.opcount(m, n, prof)
        lead = 2.0 * m * n * r - (m + n) * r * r + 2.0 / 3.0 * r ** 3
        assert abs(got - lead) <= 4.0 * (m * n + n * r + r * r)
        assert abs(got - lead) / lead < 0.02


def test_matmul_mod_helper_exact():
    """The limb-split float64 product used to build inputs equals the exact product."""
    rng = np.random.default_rng(2)
    for p in (65521, 8388593, 1073741789, 2147483647):
        X = rng.integers(0, p, size=(13, 40))
        Y = rng.integers(0, p, size=(40, 9))
        assert np.array_equal(inputs.matmul_mod(X, Y, p), exact_matmul_mod(X, Y, p))


def test_workload_generators_structure():
    """Small instances of the benchmark workloads have the promised ranks and profiles."""
    p = inputs.P_16
    A = inputs.dense_plain(m=64, n=64, r=48, p=p)
    d = oracle.cup(A, p)
    assert d["rank"] == 48 and list(d["profile"]) == list(range(48))
    p3 = inputs.P_23
    B = inputs.rank_deficient(m=140, n=60, r=40, p=p3)
    d = oracle.cup(B, p3)
    assert d["rank"] == 40
    # zeroed rows and combination rows never enter the profile
    prof = set(int(x) for x in d["profile"])
    assert all((i + 1) % 7 and (i + 1) % 5 for i in prof)
    expect = [i for i in range(140) if (i + 1) % 7 and (i + 1) % 5][:40]
    assert sorted(prof) == expect
    assert oracle.cup(inputs.dense_full(n=50, p=p), p)["rank"] == 50
    primes = inputs.primes_below(1 << 30, 64)
    assert primes[0] == 1073741789 and primes[-1] == 1073740463 and len(set(primes)) == 64
    mats = inputs.batched(count=6, lo=8, hi=24, defect=3)
    m, n, r = inputs.batched_shapes(count=6, lo=8, hi=24, defect=3)
    for b, (Ab, pb) in enumerate(mats):
        assert Ab.shape == (m[b], n[b]) and pb == primes[b % 64]
        assert oracle.cup(Ab, pb)["rank"] == r[b]


@pytest.mark.parametrize("m,n,r,p", [(5, 7, 3, 13), (20, 12, 12, 65521), (12, 20, 7, 251), (9, 9, 0, 7),
                                     (30, 30, 30, 2147483647), (6, 15, 2, 2)])
def test_oracle_nullspace_spans_the_kernel(m, n, r, p):
    """A N = 0 mod p, N has full column rank n - r (checked by the oracle's own
    elimination of N^T), and the sizes add up (rank-nullity); the zero matrix gives
    the identity."""
    from tests._helpers import exact_matmul_mod, low_rank
    rng = np.random.default_rng(m * 100 + n + r)
    A = np.zeros((m, n), dtype=np.int64) if r == 0 else (
        low_rank(rng, m, n, r, p) if r < min(m, n) else rng.integers(0, p, size=(m, n)))
    d = oracle.nullspace(A, p)
    N = d["N"].astype(np.int64)
    assert d["rank"] == r
    assert N.shape == (n, n - r)
    if n - r:
        assert not exact_matmul_mod(A, N, p).any()
        assert oracle.cup(N.T.copy(), p)["rank"] == n - r
    if r == 0:
        assert np.array_equal(N, np.eye(n, dtype=np.int64))


def _ple_parts(packed, r):
    m, n = packed.shape
    P = packed.astype(np.int64)
    L = np.zeros((m, r), dtype=np.int64)
    for t in range(r):
        L[t, t] = 1
        L[t + 1:, t] = P[t + 1:, t]
    E = np.triu(P[:r, :])
    return L, E


@pytest.mark.parametrize("m,n,r,p", [(6, 5, 3, 3), (5, 6, 4, 2), (12, 9, 9, 65521), (9, 12, 5, 251),
                                     (40, 30, 17, 2147483647)])
def test_oracle_ple_reconstructs_and_reveals_the_column_profile(m, n, r, p):
    """Exchanging rows t and ipiv[t] in order gives L E; L is unit lower, E is in row
    echelon form whose leading columns are the profile; the profile is the column
    rank profile by definition (spans of earlier columns, exhaustive for tiny p)."""
    from tests._helpers import exact_matmul_mod, low_rank, span_profile
    rng = np.random.default_rng(m + 10 * n + r)
    A = low_rank(rng, m, n, r, p) if r < min(m, n) else rng.integers(0, p, size=(m, n))
    d = oracle.ple(A, p)
    rr = d["rank"]
    assert rr == r
    L, E = _ple_parts(d["packed"], rr)
    PA = np.asarray(A, dtype=np.int64).copy()
    for t, c in enumerate(d["ipiv"]):
        PA[[t, c]] = PA[[c, t]]
    assert np.array_equal(exact_matmul_mod(L, E, p), PA % p)
    lead = [int(np.flatnonzero(E[t])[0]) for t in range(rr)]
    assert lead == list(d["profile"])
    assert all(a < b for a, b in zip(lead, lead[1:]))
    if p ** min(m, n) <= 4096:
        assert lead == span_profile(np.asarray(A).T, p)


@pytest.mark.parametrize("n,p", [(1, 7), (5, 13), (16, 65521), (23, 2147483647)])
def test_oracle_trlum_is_the_triangle_product(n, p):
    """TRLUM (Algorithm 5) against Python-integer products of the two triangles,
    taken entry by entry from the sum over k <= min(i, j)."""
    rng = np.random.default_rng(n + p % 97)
    A = rng.integers(0, p, size=(n, n))
    for unit_lower in (True, False):
        got = oracle.trlum(A, p, unit_lower)
        for i in range(n):
            for j in range(n):
                acc = 0
                for k in range(min(i, j) + 1):
                    lik = (1 if k == i else int(A[i, k])) if unit_lower else int(A[i, k])
                    ukj = int(A[k, j]) if unit_lower else (1 if k == j else int(A[k, j]))
                    acc += lik * ukj
                assert int(got[i, j]) == acc % p


@pytest.mark.parametrize("m,n,r,p", [(6, 6, 6, 7), (12, 12, 7, 65521), (9, 9, 0, 5), (10, 10, 10, 2)])
def test_oracle_trlum_rebuilds_cup(m, n, r, p):
    """The unit-U TRLUM of CUP's packed [C\\U] is A P^T (Proposition 1), also
    when A is singular (the zero blocks of the storage), and U = I, C = A
    reduces it to the identity map on a lower-triangular A."""
    rng = np.random.default_rng(m * 13 + r)
    A = low_rank(rng, m, n, r, p)
    d = oracle.cup_packed(A, p)
    Pt = perm_matrix_from_ipiv(d["ipiv"], n)
    assert np.array_equal(oracle.trlum(d["packed"], p, unit_lower=False).astype(np.int64),
                          exact_matmul_mod(A, Pt, p))
    Lw = np.tril(rng.integers(0, p, size=(m, m)))
    assert np.array_equal(oracle.trlum(Lw, p, unit_lower=False), Lw)
    Uw = np.triu(rng.integers(0, p, size=(m, m)))
    assert np.array_equal(oracle.trlum(Uw, p, unit_lower=True), Uw)


@pytest.mark.parametrize("m,n,p", [(1, 3, 7), (8, 5, 65521), (13, 13, 2147483647)])
def test_oracle_inplace_mm_is_the_product(m, n, p):
    """InPlaceMM (Algorithm 9) computes A B: exact integer product, identity and
    associativity (A (B v) = (A B) v)."""
    rng = np.random.default_rng(m + n)
    A = rng.integers(0, p, size=(m, m))
    B = rng.integers(0, p, size=(m, n))
    got = oracle.inplace_mm(A, B, p).astype(np.int64)
    assert np.array_equal(got, exact_matmul_mod(A, B, p))
    assert np.array_equal(oracle.inplace_mm(np.eye(m, dtype=np.int64), B, p).astype(np.int64), B)
    v = rng.integers(0, p, size=(n, 1))
    assert np.array_equal(exact_matmul_mod(got, v, p), exact_matmul_mod(A, exact_matmul_mod(B, v, p), p))


def _int_leibniz(M) -> int:
    n = len(M)
    total = 0
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        prod = 1
        for i in range(n):
            prod *= int(M[i][perm[i]])
        total += -prod if inv & 1 else prod
    return total


def test_oracle_int_det_against_leibniz():
    """Bareiss det over Z: every 3x3 matrix with entries in {-1, 0, 1} and random
    5x5 matrices with large signed entries, against the Leibniz formula."""
    for vals in itertools.product((-1, 0, 1), repeat=9):
        M = np.array(vals, dtype=np.int64).reshape(3, 3)
        assert oracle.int_det(M) == _int_leibniz(M)
    rng = np.random.default_rng(17)
    for n in (1, 2, 4, 5):
        for _ in range(5):
            M = rng.integers(-(1 << 40), 1 << 40, size=(n, n))
            assert oracle.int_det(M) == _int_leibniz(M)


def test_oracle_int_det_closed_forms():
    """det(L D U) = product of D for unit triangular L, U; Vandermonde =
    product of node differences; det(A B) = det A det B."""
    rng = np.random.default_rng(3)
    n = 14
    L = np.tril(rng.integers(-3, 4, size=(n, n)), -1) + np.eye(n, dtype=np.int64)
    U = np.triu(rng.integers(-3, 4, size=(n, n)), 1) + np.eye(n, dtype=np.int64)
    d = [int(x) for x in rng.integers(1, 9, size=n) * rng.choice([-1, 1], size=n)]
    A = L.astype(object).dot(np.diag(d).astype(object)).dot(U.astype(object))
    want = 1
    for x in d:
        want *= x
    assert oracle.int_det(A) == want
    x = [3, -1, 4, 10, -7, 2]
    V = np.array([[xi ** j for j in range(len(x))] for xi in x], dtype=object)
    vd = 1
    for i in range(len(x)):
        for j in range(i + 1, len(x)):
            vd *= x[j] - x[i]
    assert oracle.int_det(V) == vd
    B = rng.integers(-50, 50, size=(7, 7))
    C = rng.integers(-50, 50, size=(7, 7))
    assert oracle.int_det(B.astype(object).dot(C.astype(object))) == oracle.int_det(B) * oracle.int_det(C)


def test_oracle_int_rank_against_minors():
    """Rank over Q: the largest k with a nonzero k x k minor, by brute force on
    small matrices, and r for products of random m x r and r x n factors."""
    rng = np.random.default_rng(8)
    for _ in range(40):
        m, n = rng.integers(1, 5, size=2)
        M = rng.integers(-1, 2, size=(m, n)) * (rng.random((m, n)) < 0.6)
        best = 0
        for k in range(1, min(m, n) + 1):
            for rows in itertools.combinations(range(m), k):
                for cols in itertools.combinations(range(n), k):
                    if _int_leibniz(M[np.ix_(rows, cols)]) != 0:
                        best = k
        assert oracle.int_rank(M) == best
    X = rng.integers(-9, 10, size=(12, 4)).astype(object)
    Y = rng.integers(-9, 10, size=(4, 10)).astype(object)
    assert oracle.int_rank(X.dot(Y)) == min(4, oracle.int_rank(X), oracle.int_rank(Y))
