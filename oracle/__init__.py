"""CPU oracle for CUP over GF(p): TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check in ``__graft_entry__`` and the CPU-baseline leg
of ``bench.py`` may import this package. The product path (the CUDA library
and its Python binding) never imports, loads or calls it.

The arithmetic lives in ``cup_oracle.c`` (plain C, 64-bit integers, one
``% p`` per update, OpenMP over rows); this module builds it with gcc and
wraps it for numpy arrays. Each function cites the passage of Jeannerod,
Pernet and Storjohann it follows.

Parity status: every function is pinned by CPU tests (see tests/test_oracle_pins.py).
The values of C and U beyond their uniqueness given P are pinned by
Schur-complement minors on small matrices; the paper prints no numeric example.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cup_oracle.c")
_LIB = os.path.join(_HERE, "libcup_oracle.so")
_lock = threading.Lock()
_lib = None

_u32p = ctypes.POINTER(ctypes.c_uint32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i64 = ctypes.c_int64
_u32 = ctypes.c_uint32


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.cupo_num_threads.restype = ctypes.c_int
            L.cupo_modinv.restype = _u32
            L.cupo_modinv.argtypes = [_u32, _u32]
            L.cupo_cup.restype = _i64
            L.cupo_cup.argtypes = [_u32p, _i64, _i64, _i64, _u32, _u32p, _i64, _u32p, _i64, _i64p, _i64p]
            L.cupo_pack.restype = None
            L.cupo_pack.argtypes = [_u32p, _i64, _u32p, _i64, _i64, _i64, _i64, _u32p, _i64]
            L.cupo_laswp_cols.restype = None
            L.cupo_laswp_cols.argtypes = [_u32p, _i64, _i64, _i64p, _i64, _i64]
            L.cupo_mm_sub.restype = None
            L.cupo_mm_sub.argtypes = [_u32p, _i64, _u32p, _i64, _u32p, _i64, _i64, _i64, _i64, _u32]
            for name in ("cupo_trsm_ruu",):
                f = getattr(L, name)
                f.restype = None
                f.argtypes = [_u32p, _i64, _u32p, _i64, _i64, _i64, _u32]
            for name in ("cupo_trsm_luu", "cupo_trsm_lln"):
                f = getattr(L, name)
                f.restype = None
                f.argtypes = [_u32p, _i64, _u32p, _i64, _i64, _i64, _u32]
            L.cupo_rref.restype = _i64
            L.cupo_rref.argtypes = [_u32p, _i64, _i64, _i64, _u32, _u32p, _i64, _u32p, _i64, _i64p]
            L.cupo_det.restype = _u32
            L.cupo_det.argtypes = [_u32p, _i64, _i64, _u32]
            L.cupo_inverse.restype = ctypes.c_int
            L.cupo_inverse.argtypes = [_u32p, _i64, _i64, _u32, _u32p, _i64]
            L.cupo_solve.restype = ctypes.c_int
            L.cupo_solve.argtypes = [_u32p, _i64, _i64, _i64, _u32p, _i64, _i64, _i64p, _i64, _u32, _u32p, _i64]
            L.cupo_opcount.restype = ctypes.c_double
            L.cupo_opcount.argtypes = [_i64, _i64, _i64p, _i64]
            _lib = L
    return _lib


def _u32arr(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.uint32)


def _p32(a: np.ndarray):
    return a.ctypes.data_as(_u32p)


def _p64(a: np.ndarray):
    return a.ctypes.data_as(_i64p)


def num_threads() -> int:
    return int(lib().cupo_num_threads())


def modinv(a: int, p: int) -> int:
    """Inverse in GF(p) by the extended Euclidean algorithm (0 maps to 0)."""
    return int(lib().cupo_modinv(int(a) % p, p))


def cup(A, p: int):
    """CUP decomposition with the pivot rule of Algorithm 6 (Sec. 3.3).

    Returns dict(rank, profile, ipiv, C (m x n), U (n x n)) with A P^T = C U,
    where P^T applies the transpositions (t, ipiv[t]) to columns in order.
    """
    A = _u32arr(A)
    m, n = A.shape
    C = np.zeros((m, n), dtype=np.uint32)
    U = np.zeros((n, n), dtype=np.uint32)
    k = max(min(m, n), 1)
    ipiv = np.zeros(k, dtype=np.int64)
    prof = np.zeros(k, dtype=np.int64)
    r = lib().cupo_cup(_p32(A), m, n, n, p, _p32(C), n, _p32(U), n, _p64(ipiv), _p64(prof))
    if r < 0:
        raise MemoryError("oracle cup: allocation failed")
    return dict(rank=int(r), profile=prof[:r].copy(), ipiv=ipiv[:r].copy(), C=C, U=U)


def pack(C, U, r: int) -> np.ndarray:
    """[C\\U] space-sharing storage (Sec. 3.1)."""
    C = _u32arr(C)
    U = _u32arr(U)
    m, n = C.shape
    out = np.zeros((m, n), dtype=np.uint32)
    lib().cupo_pack(_p32(C), n, _p32(U), n, m, n, r, _p32(out), n)
    return out


def cup_packed(A, p: int):
    """CUP with the result in [C\\U] storage, as Algorithm 6 leaves it in A."""
    d = cup(A, p)
    d["packed"] = pack(d["C"], d["U"], d["rank"])
    return d


def laswp_cols(A, ipiv, k0: int = 0, k1: int | None = None) -> np.ndarray:
    """A P^T for the transpositions (t, ipiv[t]), t = k0..k1-1, applied in order."""
    A = _u32arr(A).copy()
    ipiv = np.ascontiguousarray(ipiv, dtype=np.int64)
    if k1 is None:
        k1 = len(ipiv)
    m, n = A.shape
    full = np.arange(max(n, 1), dtype=np.int64)
    full[: len(ipiv)] = ipiv
    lib().cupo_laswp_cols(_p32(A), m, n, _p64(full), k0, k1)
    return A


def mm_sub(Cm, A, B, p: int) -> np.ndarray:
    """Algorithm 1 with alpha = -1, beta = 1: returns C - A B mod p."""
    Cm = _u32arr(Cm).copy()
    A = _u32arr(A)
    B = _u32arr(B)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2 and Cm.shape == (M, N)
    lib().cupo_mm_sub(_p32(Cm), N, _p32(A), max(K, 1), _p32(B), max(N, 1), M, N, K, p)
    return Cm


def matmul(A, B, p: int) -> np.ndarray:
    """A B mod p (Algorithm 1 with alpha = 1 on a zero C: the negation of 0 - A B)."""
    A = _u32arr(A)
    B = _u32arr(B)
    neg = mm_sub(np.zeros((A.shape[0], B.shape[1]), dtype=np.uint32), A, B, p).astype(np.uint64)
    return ((p - neg) % p).astype(np.uint32)


def trlum(A, p: int, unit_lower: bool = True) -> np.ndarray:
    """TRLUM (Algorithm 5) by its definition: A = [L\\U] -> L U.

    unit_lower: L has the implicit unit diagonal and U keeps the stored one
    (Algorithm 5 as stated); otherwise U is unit and L carries the diagonal,
    as in the [C\\U] factors of CUP (Algorithm 9)."""
    A = _u32arr(A)
    n = A.shape[0]
    eye = np.eye(n, dtype=np.uint32)
    if unit_lower:
        L, U = np.tril(A, -1) + eye, np.triu(A)
    else:
        L, U = np.tril(A), np.triu(A, 1) + eye
    return matmul(L, U, p)


def inplace_mm(A, B, p: int) -> np.ndarray:
    """InPlaceMM (Algorithm 9) by what it computes: A B mod p."""
    return matmul(A, B, p)


def trsm_right_upper_unit(U, B, p: int) -> np.ndarray:
    """TRSM(Right, Upper, Unit): B U^{-1} (Algorithm 2, unit-diagonal variant)."""
    U = _u32arr(U)
    B = _u32arr(B).copy()
    m, n = B.shape
    lib().cupo_trsm_ruu(_p32(U), U.shape[1], _p32(B), max(n, 1), m, n, p)
    return B


def trsm_left_upper_unit(U, B, p: int) -> np.ndarray:
    """TRSM(Left, Upper, Unit): U^{-1} B."""
    U = _u32arr(U)
    B = _u32arr(B).copy()
    n, k = B.shape
    lib().cupo_trsm_luu(_p32(U), U.shape[1], _p32(B), max(k, 1), n, k, p)
    return B


def trsm_left_lower_nonunit(L, B, p: int) -> np.ndarray:
    """TRSM(Left, Lower, NonUnit): L^{-1} B."""
    L = _u32arr(L)
    B = _u32arr(B).copy()
    n, k = B.shape
    lib().cupo_trsm_lln(_p32(L), L.shape[1], _p32(B), max(k, 1), n, k, p)
    return B


def rref(A, p: int, want_x: bool = False):
    """Reduced column echelon form R (Proposition 1) by column Gauss-Jordan.

    Returns dict(rank, profile, R, X) with A X = R (X is None unless asked)."""
    A = _u32arr(A)
    m, n = A.shape
    R = np.zeros((m, n), dtype=np.uint32)
    X = np.zeros((n, n), dtype=np.uint32) if want_x else None
    prof = np.zeros(max(min(m, n), 1), dtype=np.int64)
    xp = _p32(X) if want_x else ctypes.cast(None, _u32p)
    r = lib().cupo_rref(_p32(A), m, n, n, p, _p32(R), n, xp, n, _p64(prof))
    return dict(rank=int(r), profile=prof[:r].copy(), R=R, X=X)


def ple(A, p: int):
    """PLE decomposition (Sec. 5): (E^T, L^T, P^T) is the CUP decomposition of A^T,
    so this is `cup_packed` of A^T, transposed. Returns dict(rank, profile (the column
    rank profile), ipiv (row exchanges), packed = [L\\E] as an m x n array)."""
    A = _u32arr(A)
    d = cup_packed(np.ascontiguousarray(A.T), p)
    return dict(rank=d["rank"], profile=d["profile"], ipiv=d["ipiv"],
                packed=np.ascontiguousarray(d["packed"].T))


def nullspace(A, p: int):
    """Basis of the right nullspace {x : A x = 0}: with A X = R (the reduced column
    echelon transform of `rref`), R's columns r .. n-1 vanish, so X's columns r .. n-1
    are a basis (Sec. 3.4, 3.5 and 4.4). Returns dict(rank, N) with N of shape (n, n - r)."""
    d = rref(A, p, want_x=True)
    r = d["rank"]
    return dict(rank=r, N=np.ascontiguousarray(d["X"][:, r:]))


def det(A, p: int) -> int:
    """Determinant by row-echelon elimination with interchanges."""
    A = _u32arr(A)
    n = A.shape[0]
    assert A.shape == (n, n)
    return int(lib().cupo_det(_p32(A), n, n, p))


def inverse(A, p: int):
    """A^{-1} by Gauss-Jordan on [A | I]; None if A is singular."""
    A = _u32arr(A)
    n = A.shape[0]
    out = np.zeros((n, n), dtype=np.uint32)
    s = lib().cupo_inverse(_p32(A), n, n, p, _p32(out), n)
    return None if s else out


def solve(A, B, p: int):
    """Solution of A X = B supported on the CUP pivot columns (zero elsewhere).

    Returns (status, X, rank): status 0 = solved, 2 = inconsistent."""
    A = _u32arr(A)
    B = _u32arr(B)
    if B.ndim == 1:
        B = B[:, None]
    m, n = A.shape
    k = B.shape[1]
    d = cup(A, p)
    X = np.zeros((n, k), dtype=np.uint32)
    ipiv = np.ascontiguousarray(d["ipiv"], dtype=np.int64)
    if ipiv.size == 0:
        ipiv = np.zeros(1, dtype=np.int64)
    s = lib().cupo_solve(_p32(A), m, n, n, _p32(B), k, k, _p64(ipiv), d["rank"], p, _p32(X), k)
    return int(s), X, d["rank"]


def int_det(A) -> int:
    """det of an integer matrix over Z by fraction-free (Bareiss) elimination on
    Python integers: exact, for the small sizes the tests use. It is the value
    the multi-modular path must reconstruct (Sec. 1: integer problems reduced to
    prime fields)."""
    M = [[int(x) for x in row] for row in np.asarray(A)]
    n = len(M)
    if n == 0:
        return 1
    sign, prev = 1, 1
    for k in range(n - 1):
        if M[k][k] == 0:
            sw = next((i for i in range(k + 1, n) if M[i][k] != 0), None)
            if sw is None:
                return 0
            M[k], M[sw] = M[sw], M[k]
            sign = -sign
        for i in range(k + 1, n):
            for j in range(k + 1, n):
                M[i][j] = (M[i][j] * M[k][k] - M[i][k] * M[k][j]) // prev
        prev = M[k][k]
    return sign * M[n - 1][n - 1]


def int_rank(A) -> int:
    """rank over Q of an integer matrix: Gaussian elimination on exact rationals
    (Python fractions), for the small sizes the tests use."""
    from fractions import Fraction
    M = [[Fraction(int(x)) for x in row] for row in np.asarray(A)]
    m = len(M)
    n = len(M[0]) if m else 0
    r = 0
    for c in range(n):
        piv = next((i for i in range(r, m) if M[i][c] != 0), None)
        if piv is None:
            continue
        M[r], M[piv] = M[piv], M[r]
        for i in range(r + 1, m):
            if M[i][c]:
                f = M[i][c] / M[r][c]
                M[i] = [x - f * y for x, y in zip(M[i], M[r])]
        r += 1
        if r == m:
            break
    return r


def opcount(m: int, n: int, profile) -> float:
    prof = np.ascontiguousarray(profile, dtype=np.int64)
    if prof.size == 0:
        return 0.0
    return float(lib().cupo_opcount(m, n, _p64(prof), prof.size))


def perm_from_ipiv(ipiv, n: int) -> np.ndarray:
    """Position -> original column after applying transpositions (t, ipiv[t]) in order:
    (A P^T)[:, q] = A[:, perm[q]]."""
    perm = np.arange(n, dtype=np.int64)
    for t, c in enumerate(ipiv):
        perm[t], perm[c] = perm[c], perm[t]
    return perm
