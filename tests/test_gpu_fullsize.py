"""Parity at the benchmark workloads' full sizes, element by element against the oracle.

The oracle's results at these sizes are stored as SHA-256 digests in
tests/golden/fullsize_digests.json, written by tests/golden/make_fullsize_digests.py,
which calls only the oracle and the input generators (the oracle needs minutes per
case on the host). Each test computes the same digest of the CUDA path's output:
equal digests mean equal arrays. The input's digest is checked first, so that a
difference in input generation is reported as such. The CUDA calls run in the launch
configuration bench.py times (tensor engine, default options, repeated calls on a
stream of our own, so the second call is a CUDA-graph replay; the host-buffer entry
point of the end-to-end leg).

Before the digests, a cheap check that holds at any size runs too (and is the only
element-wise check for the 32768^2 workload, whose oracle would need hours):
  * [C\\U] has the shape the decomposition promises (Proposition 1): C in
    column echelon form with nonzero pivots at the reported row rank profile,
    zeros outside C and U, the transpositions in LAPACK form (ipiv[t] >= t);
  * A P^T = C U, by Freivalds' test with random vectors modulo p (a wrong entry
    anywhere survives one vector with probability at most 1/p), evaluated
    exactly in 64-bit integer blocks.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1112_5717_gb300 import inputs
from tests.golden.make_fullsize_digests import digest

_GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize_digests.json")

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


def _golden(case):
    data = json.load(open(_GOLDEN))
    if case not in data:
        pytest.fail(f"{case}: no oracle digest in {_GOLDEN} (run tests/golden/make_fullsize_digests.py)")
    return data[case]


def _check_input(rec, *arrays):
    assert digest(*arrays) == rec["input"], "the input generator made a different matrix than the oracle's run"


def _check_cup(rec, r, prof, ipiv, packed):
    want = rec["cup"]
    assert r == want["rank"]
    assert digest(np.asarray(prof[:r], dtype=np.int64)) == want["profile"], "row rank profile differs from the oracle"
    assert digest(np.asarray(ipiv[:r], dtype=np.int64)) == want["ipiv"], "transpositions differ from the oracle"
    assert digest(packed) == want["packed"], "[C\\U] differs from the oracle"


def _factor_like_bench(cup, A, p):
    """Two calls as bench.py makes them (tensor engine, default options, a stream of
    our own: the second is a graph replay); returns the host result of the second."""
    import torch
    u8 = A.dtype == np.uint8
    h = cup.Handle(engine=cup.ENGINE_TENSOR)
    src = torch.from_numpy(A.copy() if u8 else np.ascontiguousarray(A, dtype=np.uint32).view(np.int32)).cuda()
    work = torch.empty_like(src)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    outs = []

    def host(t):
        return t.cpu().numpy().copy() if u8 else t.cpu().numpy().view(np.uint32).copy()

    with torch.cuda.stream(stream):
        for _ in range(2):
            work.copy_(src)
            r, prof, ipiv = h.factor(work, p)
            torch.cuda.synchronize()
            outs.append((r, prof[:r].cpu().numpy(), ipiv[:r].cpu().numpy(), host(work)))
    # the host-buffer entry point of the end-to-end leg, also replayed on its second call
    hA = src.cpu().pin_memory()
    hout = torch.empty_like(hA).pin_memory()
    with torch.cuda.stream(stream):
        for _ in range(2):
            rh, _, _ = h.factor_host(hA, work, p, out=hout)
    torch.cuda.synchronize()
    h.close()
    return outs, rh, (hout.numpy().copy() if u8 else hout.numpy().view(np.uint32))


def _run_factor(cuda_lib, case, A, p):
    rec = _golden(case)
    _check_input(rec, A)
    outs, rh, hout = _factor_like_bench(cuda_lib, A, p)
    (r0, prof0, ipiv0, P0), (r1, prof1, ipiv1, P1) = outs
    # the replayed call reproduces the first one exactly, and so does the host-buffer call
    assert r0 == r1 == rh
    assert np.array_equal(prof0, prof1) and np.array_equal(ipiv0, ipiv1) and np.array_equal(P0, P1)
    assert np.array_equal(hout, P1)
    check_cup_at_scale(A, P1, prof1, ipiv1, r1, p)
    _check_cup(rec, r1, prof1, ipiv1, P1)
    return rec


def test_full_size_dense_8192(cuda_lib):
    _run_factor(cuda_lib, "dense_full_8192", inputs.dense_full(n=8192, p=inputs.P_16), inputs.P_16)


def test_full_size_rank_deficient(cuda_lib):
    rec = _run_factor(cuda_lib, "rank_deficient", inputs.rank_deficient(p=inputs.P_23), inputs.P_23)
    assert rec["cup"]["rank"] <= 3000


def test_full_size_small_p_8192_u8(cuda_lib):
    """The 32768^2 GF(251) workload's structure (one centred 8-bit limb, one-byte
    storage) at 8192^2, where the oracle finishes."""
    _run_factor(cuda_lib, "dense_small_p_8192", inputs.dense_small_p(n=8192, p=inputs.P_8), inputs.P_8)


def _freivalds_inverse(A, Ainv, p, trials):
    """A (A^{-1} x) = x for random x modulo p."""
    rng = np.random.default_rng(7)
    for _ in range(trials):
        x = rng.integers(0, p, size=A.shape[1], dtype=np.int64)
        y = _matvec_mod(A, _matvec_mod(Ainv, x, p), p)
        assert np.array_equal(y, x), "A A^-1 != I"


@pytest.mark.parametrize("case", ["dense_full_8192", "dense_small_p_8192"])
def test_full_size_det_and_inverse(cuda_lib, case):
    import torch
    if case == "dense_full_8192":
        A, p = inputs.dense_full(n=8192, p=inputs.P_16), inputs.P_16
        dev = torch.from_numpy(A.view(np.int32).copy()).cuda()
        host = lambda t: t.cpu().numpy().view(np.uint32)          # noqa: E731
    else:
        A, p = inputs.dense_small_p(n=8192, p=inputs.P_8), inputs.P_8
        dev = torch.from_numpy(A.copy()).cuda()
        host = lambda t: t.cpu().numpy()                           # noqa: E731
    rec = _golden(case)
    _check_input(rec, A)
    h = cuda_lib.Handle(engine=cuda_lib.ENGINE_TENSOR)
    work = dev.clone()
    assert h.det(work, p) == rec["det"], "determinant differs from the oracle"
    work.copy_(dev)
    assert h.inverse(work, p) == (rec["inverse"] is not None)
    inv = host(work)
    _freivalds_inverse(A, inv, p, trials=max(2, -(-30 // max(1, int(np.log2(p))))))
    assert digest(inv) == rec["inverse"], "inverse differs from the oracle"
    h.close()


def test_full_size_rref(cuda_lib):
    """Reduced column echelon form R and its transform X of the 16384 x 4096 workload."""
    import torch
    A, p = inputs.rank_deficient(p=inputs.P_23), inputs.P_23
    rec = _golden("rank_deficient")
    _check_input(rec, A)
    h = cuda_lib.Handle(engine=cuda_lib.ENGINE_TENSOR)
    dA = torch.from_numpy(A.view(np.int32).copy()).cuda()
    r, prof, X = h.rref(dA, p, want_x=True)
    want = rec["rref"]
    assert r == want["rank"]
    assert digest(prof[:r].cpu().numpy().astype(np.int64)) == want["profile"]
    assert digest(dA.cpu().numpy().view(np.uint32)) == want["R"], "R differs from the oracle"
    assert digest(X.cpu().numpy().view(np.uint32)) == want["X"], "X differs from the oracle"
    h.close()


def test_full_size_batched(cuda_lib):
    """All 4096 matrices of the batched workload, each modulo its own prime near 2^30,
    in the one launch bench.py times: rank, [C\\U], profile, transpositions and, for the
    square ones, the determinant of every matrix."""
    import torch
    mats = inputs.batched()
    rec = _golden("batched")
    _check_input(rec, *[A for A, _ in mats])
    h = cuda_lib.Handle()
    dm = [torch.from_numpy(np.ascontiguousarray(A, dtype=np.uint32).view(np.int32)).cuda() for A, _ in mats]
    ranks, profs, ipivs, dets = h.factor_batched(dm, [q for _, q in mats], want_det=True)
    torch.cuda.synchronize()
    ranks = ranks.cpu().numpy().tolist()
    dets = dets.cpu().numpy().view(np.uint32)
    assert ranks == rec["ranks"], [b for b, (x, y) in enumerate(zip(ranks, rec["ranks"])) if x != y][:10]
    bad = []
    for b, (A, q) in enumerate(mats):
        r = ranks[b]
        dg = digest(dm[b].cpu().numpy().view(np.uint32), profs[b][:r].cpu().numpy().astype(np.int64),
                    ipivs[b][:r].cpu().numpy().astype(np.int64))[:16]
        if dg != rec["cup"][b]:
            bad.append(b)
        if rec["det"][b] is not None and int(dets[b]) != rec["det"][b]:
            bad.append(b)
    assert not bad, f"matrices differing from the oracle: {sorted(set(bad))[:20]}"
    h.close()


def test_full_size_small_p_32768_u8(cuda_lib):
    """The 32768^2 GF(251) workload itself (one-byte storage, as bench.py times it):
    shape of [C\\U] and Freivalds' test of A P^T = C U, the replayed and host-buffer
    calls equal to the first; the oracle would need hours here, so its element-wise
    comparison is the 8192^2 case above."""
    A, p = inputs.dense_small_p(n=32768, p=inputs.P_8), inputs.P_8
    outs, rh, hout = _factor_like_bench(cuda_lib, A, p)
    (r0, prof0, ipiv0, P0), (r1, prof1, ipiv1, P1) = outs
    assert r0 == r1 == rh
    assert np.array_equal(prof0, prof1) and np.array_equal(ipiv0, ipiv1) and np.array_equal(P0, P1)
    assert np.array_equal(hout, P1)
    check_cup_at_scale(A, P1, prof1, ipiv1, r1, p, trials=5)
