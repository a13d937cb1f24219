"""Parity at the benchmark's full sizes, in the launch configuration bench.py times
(tensor engine, default options, repeated calls on a stream of our own, so the
second call is a CUDA-graph replay; the host-buffer entry point as in the
end-to-end leg).

The oracle cannot factor these sizes in test time, so the result is checked by
properties that hold at any size and pin it down:
  * [C\\U] has the shape the decomposition promises (Proposition 1): C in
    column echelon form with nonzero pivots at the reported row rank profile,
    zeros outside C and U, the transpositions in LAPACK form (ipiv[t] >= t);
  * A P^T = C U, by Freivalds' test with random vectors modulo p (a wrong entry
    anywhere survives one vector with probability at most 1/p), evaluated
    exactly in 64-bit integer blocks.
Together these make the rank and the row rank profile exact (the row rank profile
of A P^T = C U is that of C, whose pivot rows are the reported profile).
"""
import numpy as np
import pytest

import oracle
from paper_1112_5717_gb300 import inputs

pytestmark = pytest.mark.gpu

_BLK = 1024   # column block of the exact products: 1024 (p - 1)^2 < 2^63 for p < 2^26


def _matvec_mod(M, x, p, col_mask=None):
    """(M x) mod p exactly, M (rows x cols) any integer array, in column blocks;
    col_mask(j0, j1) may give a boolean mask (rows x (j1 - j0)) selecting the
    entries of M that are part of the matrix."""
    rows, cols = M.shape
    out = np.zeros(rows, dtype=np.int64)
    x = np.asarray(x, dtype=np.int64)
    for j0 in range(0, cols, _BLK):
        j1 = min(cols, j0 + _BLK)
        blk = M[:, j0:j1].astype(np.int64)
        if col_mask is not None:
            blk *= col_mask(j0, j1)
        out = (out + (blk @ x[j0:j1]) % p) % p
    return out


def check_cup_at_scale(A, packed, prof, ipiv, r, p, trials=None, seed=12):
    """Structure of [C\\U] and A P^T = C U (Freivalds) for an m x n result of rank r;
    enough random vectors that a wrong result passes with probability below 2^-30."""
    m, n = A.shape
    if trials is None:
        trials = max(2, -(-30 // max(1, int(np.log2(p)))))
    prof = np.asarray(prof[:r], dtype=np.int64)
    ipiv = np.asarray(ipiv[:r], dtype=np.int64)
    assert r <= min(m, n)
    assert np.all(np.diff(prof) > 0) and (r == 0 or (prof[0] >= 0 and prof[-1] < m))
    assert np.all(ipiv >= np.arange(r)) and np.all(ipiv < n)
    rows = np.arange(m)[:, None]
    # C: column k holds its pivot at row prof[k] (nonzero) and zeros in rows k .. prof[k] - 1
    assert np.all(packed[prof, np.arange(r)] != 0)
    for k0 in range(0, r, _BLK):
        k1 = min(r, k0 + _BLK)
        ks = np.arange(k0, k1)[None, :]
        above = (rows >= ks) & (rows < prof[k0:k1][None, :])
        assert not np.any(packed[:, k0:k1][above])
    # outside C (columns < r) and U (rows < r) the storage is zero
    assert not np.any(packed[r:, r:])
    perm = oracle.perm_from_ipiv(ipiv, n)                # (A P^T)[:, q] = A[:, perm[q]]
    urows = np.arange(r)[:, None]
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        x = rng.integers(0, p, size=n, dtype=np.int64)
        z = np.zeros(n, dtype=np.int64)
        z[perm] = x
        y1 = _matvec_mod(A, z, p)                        # (A P^T) x
        # U x with U = [unit diagonal | strict upper part of rows 0 .. r-1]
        ux = (x[:r] + _matvec_mod(packed[:r], x, p,
                                  lambda j0, j1: np.arange(j0, j1)[None, :] > urows)) % p
        # C (U x) with C = the part of columns 0 .. r-1 on and below the diagonal
        y2 = _matvec_mod(packed[:, :r], ux, p, lambda k0, k1: rows >= np.arange(k0, k1)[None, :])
        assert np.array_equal(y1, y2)


def _factor_like_bench(cup, A, p):
    """Two calls as bench.py makes them (tensor engine, default options, a stream of
    our own: the second is a graph replay); returns the host result of the second."""
    import torch
    h = cup.Handle(engine=cup.ENGINE_TENSOR)
    src = torch.from_numpy(np.ascontiguousarray(A, dtype=np.uint32).view(np.int32)).cuda()
    work = torch.empty_like(src)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    outs = []
    with torch.cuda.stream(stream):
        for _ in range(2):
            work.copy_(src)
            r, prof, ipiv = h.factor(work, p)
            torch.cuda.synchronize()
            outs.append((r, prof[:r].cpu().numpy(), ipiv[:r].cpu().numpy(),
                         work.cpu().numpy().view(np.uint32).copy()))
    # the host-buffer entry point of the end-to-end leg, also replayed on its second call
    hA = torch.from_numpy(np.ascontiguousarray(A, dtype=np.uint32).view(np.int32)).pin_memory()
    hout = torch.empty_like(hA).pin_memory()
    with torch.cuda.stream(stream):
        for _ in range(2):
            rh, _, _ = h.factor_host(hA, work, p, out=hout)
    torch.cuda.synchronize()
    h.close()
    return outs, rh, hout.numpy().view(np.uint32)


@pytest.mark.parametrize("workload", ["dense_full_8192", "rank_deficient_16384x4096"])
def test_full_size_factorization(cuda_lib, workload):
    if workload == "dense_full_8192":
        A, p = inputs.dense_full(n=8192, p=inputs.P_16), inputs.P_16
    else:
        A, p = inputs.rank_deficient(p=inputs.P_23), inputs.P_23
    outs, rh, hout = _factor_like_bench(cuda_lib, A, p)
    (r0, prof0, ipiv0, P0), (r1, prof1, ipiv1, P1) = outs
    # the replayed call reproduces the first one exactly, and so does the host-buffer call
    assert r0 == r1 == rh
    assert np.array_equal(prof0, prof1) and np.array_equal(ipiv0, ipiv1) and np.array_equal(P0, P1)
    assert np.array_equal(hout, P1)
    check_cup_at_scale(A, P1, prof1, ipiv1, r1, p)
    if workload == "rank_deficient_16384x4096":
        assert r1 <= 3000
