"""Batched multi-modular CUP: every matrix of a batch, each over its own
prime, matches the oracle's factors, rank, profile, transpositions and (for
square ones) determinant."""
import numpy as np
import pytest

import oracle
from paper_1112_5717_gb300 import inputs

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("count,lo,hi,defect", [(40, 8, 96, 4), (12, 64, 300, 32)])
def test_batched_matches_oracle(cuda_lib, count, lo, hi, defect):
    import torch
    mats = inputs.batched(count=count, lo=lo, hi=hi, defect=defect, seed=inputs.SEED_BASE + 50 + count)
    # a few square items, a few with forced transpositions, one tiny prime
    extra = [(inputs.dense_full(n=33, p=65521, seed=3), 65521), (inputs.dense_full(m=20, n=45, p=3, seed=4), 3),
             (np.zeros((17, 9), dtype=np.uint32), 1073741789)]
    mats = mats + extra
    h = cuda_lib.Handle()
    dmats = [_dev(A) for A, _ in mats]
    ranks, profs, ipivs, dets = h.factor_batched(dmats, [p for _, p in mats], want_det=True)
    torch.cuda.synchronize()
    ranks = ranks.cpu().numpy()
    dets = dets.cpu().numpy().view(np.uint32)
    for b, (A, p) in enumerate(mats):
        want = oracle.cup_packed(A, p)
        r = want["rank"]
        assert ranks[b] == r, b
        assert np.array_equal(profs[b][:r].cpu().numpy(), want["profile"]), b
        assert np.array_equal(ipivs[b][:r].cpu().numpy(), want["ipiv"]), b
        assert np.array_equal(_host(dmats[b]), want["packed"]), b
        if A.shape[0] == A.shape[1]:
            assert dets[b] == oracle.det(A, p), b


def test_batched_flags_invalid_items(cuda_lib):
    import torch
    A = inputs.dense_full(n=20, p=65521)
    h = cuda_lib.Handle()
    dA, dB = _dev(A), _dev(A)
    ranks, _, _, _ = h.factor_batched([dA, dB], [65521, 65520])      # 65520 is not prime
    torch.cuda.synchronize()
    r = ranks.cpu().numpy()
    assert r[0] == 20 and r[1] == -1
