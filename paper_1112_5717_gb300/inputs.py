"""Seeded synthetic input generators for CUP over GF(p).

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests. It holds no step of the CUP method: it only draws random
residues and builds structured test matrices (products X*Y mod p, zeroed rows,
linear-combination rows) with numpy's PCG64 generator.

The workloads mirror the shapes the paper's analysis is about (Sec. 4.2: an
m x n matrix of rank r, dense, rectangular or rank deficient) at five
configurations:

  dense_plain      512 x 512, GF(65521), rank 384 = (512x384)(384x512), rows shuffled
  dense_full       8192 x 8192, GF(65521), uniform entries (full rank w.h.p.)
  rank_deficient   16384 x 4096, GF(8388593), rank 3000 = X*Y, every 7th row zeroed,
                   every 5th row a random combination of 4 earlier rows
  dense_small_p    32768 x 32768, GF(251), uniform entries (uint8 storage)
  batched          4096 matrices, m, n log-uniform in [64, 1024], rank min(m,n) - U{0..32},
                   each modulo its own prime among the 64 largest primes below 2^30

Every generator takes its sizes as arguments so that tests can draw the same
structure at sizes the oracle finishes in seconds.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 11112

P_16 = 65521          # largest prime below 2^16
P_23 = 8388593        # largest prime below 2^23
P_8 = 251             # largest prime below 2^8


def _is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (bases 2..37)."""
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for q in small:
        if n % q == 0:
            return n == q
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def is_prime(n: int) -> bool:
    return _is_prime(int(n))


def primes_below(bound: int, count: int) -> list[int]:
    """The `count` largest primes strictly below `bound`, in decreasing order."""
    out = []
    n = bound - 1
    while len(out) < count:
        if _is_prime(n):
            out.append(n)
        n -= 1
    return out


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform(rng: np.random.Generator, m: int, n: int, p: int, dtype=np.uint32) -> np.ndarray:
    """m x n matrix with entries uniform in [0, p)."""
    return rng.integers(0, p, size=(m, n), dtype=np.int64).astype(dtype)


def matmul_mod(X: np.ndarray, Y: np.ndarray, p: int) -> np.ndarray:
    """Exact (X @ Y) mod p for residues below 2^31, via 16-bit limbs in float64.

    Each partial product has entries below 2^16 * 2^16 = 2^32 summed over at
    most 2^20 terms, so every float64 partial sum is an exact integer below
    2^52; the limbs are then recombined modulo p with int64 arithmetic.
    """
    X = np.asarray(X, dtype=np.int64)
    Y = np.asarray(Y, dtype=np.int64)
    assert X.shape[1] == Y.shape[0] and X.shape[1] <= (1 << 20)
    x0, x1 = (X & 0xFFFF).astype(np.float64), (X >> 16).astype(np.float64)
    y0, y1 = (Y & 0xFFFF).astype(np.float64), (Y >> 16).astype(np.float64)
    s00 = np.asarray(x0 @ y0).astype(np.int64) % p
    s01 = (np.asarray(x0 @ y1).astype(np.int64) + np.asarray(x1 @ y0).astype(np.int64)) % p
    s11 = np.asarray(x1 @ y1).astype(np.int64) % p
    t16 = (1 << 16) % p
    t32 = (1 << 32) % p
    out = (s00 + (s01 * t16) % p + (s11 * t32) % p) % p
    return out


def dense_plain(m: int = 512, n: int = 512, r: int = 384, p: int = P_16, seed: int = SEED_BASE + 1):
    """A = X*Y mod p (X m x r, Y r x n uniform), rows shuffled by a seeded permutation."""
    rng = rng_for(seed)
    X = uniform(rng, m, r, p, np.int64)
    Y = uniform(rng, r, n, p, np.int64)
    A = matmul_mod(X, Y, p)
    A = A[rng.permutation(m)]
    return A.astype(np.uint32)


def dense_full(n: int = 8192, p: int = P_16, seed: int = SEED_BASE + 2, m: int | None = None):
    """m x n (default square) uniform residues: full rank with probability ~ 1 - 1/p."""
    rng = rng_for(seed)
    return uniform(rng, n if m is None else m, n, p, np.uint32)


def rank_deficient(m: int = 16384, n: int = 4096, r: int = 3000, p: int = P_23,
                   seed: int = SEED_BASE + 3, zero_every: int = 7, comb_every: int = 5,
                   comb_terms: int = 4):
    """A = X*Y mod p of rank <= r; then, for 0-based row i in increasing order,
    row i is zeroed if (i+1) % zero_every == 0, else replaced by a random
    combination of `comb_terms` earlier rows (coefficients uniform in [1, p)) if
    (i+1) % comb_every == 0."""
    rng = rng_for(seed)
    X = uniform(rng, m, r, p, np.int64)
    Y = uniform(rng, r, n, p, np.int64)
    A = matmul_mod(X, Y, p)
    for i in range(m):
        if (i + 1) % zero_every == 0:
            A[i] = 0
        elif (i + 1) % comb_every == 0 and i >= 1:
            rows = rng.integers(0, i, size=comb_terms)
            coef = rng.integers(1, p, size=comb_terms, dtype=np.int64)
            acc = np.zeros(n, dtype=np.int64)
            for rr, cc in zip(rows, coef):
                acc = (acc + cc * A[rr]) % p
            A[i] = acc
    return A.astype(np.uint32)


def dense_small_p(n: int = 32768, p: int = P_8, seed: int = SEED_BASE + 4):
    """n x n uniform residues modulo a prime below 2^8, stored as uint8."""
    rng = rng_for(seed)
    return uniform(rng, n, n, p, np.uint8)


def batched_shapes(count: int = 4096, lo: int = 64, hi: int = 1024, defect: int = 32,
                   seed: int = SEED_BASE + 5):
    """(m, n, r) triples: m, n = round(exp(U[ln lo, ln hi])) independently and
    r = min(m, n) - U{0..defect} (clamped at 0)."""
    rng = rng_for(seed)
    m = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)
    n = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)
    d = rng.integers(0, defect + 1, size=count)
    r = np.maximum(np.minimum(m, n) - d, 0)
    return m, n, r


def batched(count: int = 4096, lo: int = 64, hi: int = 1024, defect: int = 32,
            nprimes: int = 64, seed: int = SEED_BASE + 5):
    """List of (A_b, p_b): A_b = X_b * Y_b mod p_b with X_b m x r, Y_b r x n,
    p_b = primes[b mod nprimes] where primes are the largest primes below 2^30."""
    m, n, r = batched_shapes(count, lo, hi, defect, seed)
    primes = primes_below(1 << 30, nprimes)
    rng = rng_for(seed + 7919)
    out = []
    for b in range(count):
        p = primes[b % nprimes]
        X = uniform(rng, int(m[b]), int(r[b]), p, np.int64)
        Y = uniform(rng, int(r[b]), int(n[b]), p, np.int64)
        A = matmul_mod(X, Y, p) if r[b] > 0 else np.zeros((m[b], n[b]), dtype=np.int64)
        out.append((A.astype(np.uint32), p))
    return out
