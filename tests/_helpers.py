"""Independent arithmetic used by the tests to pin the oracle and the CUDA path.

Everything here uses Python integers (exact, arbitrary precision) or textbook
definitions (Leibniz determinant, span enumeration), not the oracle's code.
"""
from __future__ import annotations

import itertools

import numpy as np


def leibniz_det(M, p: int) -> int:
    """det(M) mod p by the Leibniz formula (sum over permutations)."""
    M = [[int(x) for x in row] for row in M]
    n = len(M)
    if n == 0:
        return 1 % p
    total = 0
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        prod = 1
        for i in range(n):
            prod = prod * M[i][perm[i]] % p
        total += -prod if inv & 1 else prod
    return total % p


def exact_matmul_mod(A, B, p: int) -> np.ndarray:
    """(A @ B) mod p with Python integers (object arrays): exact at any size."""
    Ao = np.asarray(A, dtype=np.int64).astype(object)
    Bo = np.asarray(B, dtype=np.int64).astype(object)
    return (Ao.dot(Bo) % p).astype(np.int64)


def perm_matrix_from_ipiv(ipiv, n: int) -> np.ndarray:
    """Pt such that (A @ Pt) applies the transpositions (t, ipiv[t]) to A's
    columns in order t = 0, 1, ... (Pt = T_0 T_1 ... as column operations)."""
    Pt = np.eye(n, dtype=np.int64)
    for t, c in enumerate(ipiv):
        T = np.eye(n, dtype=np.int64)
        T[[t, c]] = T[[c, t]]
        Pt = Pt @ T
    return Pt


def span_profile(A, p: int):
    """Row rank profile by definition (Sec. 2): row i is in the profile iff it
    is not in the span of the earlier rows; spans enumerated exhaustively."""
    A = np.asarray(A, dtype=np.int64) % p
    m, n = A.shape
    span = {tuple([0] * n)}
    prof = []
    for i in range(m):
        v = tuple(int(x) for x in A[i])
        if v in span:
            continue
        prof.append(i)
        new = set()
        for s in span:
            for c in range(p):
                new.add(tuple((s[j] + c * v[j]) % p for j in range(n)))
        span = new
    return prof


def random_invertible(rng, n: int, p: int) -> np.ndarray:
    """L * U with random unit lower L and unit upper U: always invertible."""
    L = np.tril(rng.integers(0, p, size=(n, n)), -1) + np.eye(n, dtype=np.int64)
    U = np.triu(rng.integers(0, p, size=(n, n)), 1) + np.eye(n, dtype=np.int64)
    return exact_matmul_mod(L, U, p)


def low_rank(rng, m: int, n: int, r: int, p: int) -> np.ndarray:
    X = rng.integers(0, p, size=(m, r))
    Y = rng.integers(0, p, size=(r, n))
    return exact_matmul_mod(X, Y, p)
