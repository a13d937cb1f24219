"""One-byte residue storage (p < 2^8) against the oracle, element by element.

The *_u8 entry points take uint8 matrices; the results (packed [C\\U], profile,
pivots, rank, determinant, inverse) must equal the oracle's on the same values, on
both engines, for square, rectangular, rank-deficient and ragged shapes (widths that
are not a multiple of 16 take the kernels' unvectorised tails), with a padded leading
dimension, on repeated calls (the second is a CUDA-graph replay) and through the
host-buffer call.
"""
import numpy as np
import pytest

import oracle
from paper_1112_5717_gb300 import inputs

from _helpers import low_rank

pytestmark = pytest.mark.gpu

P = inputs.P_8


def _cases():
    rng = np.random.default_rng(251)
    dense = inputs.dense_small_p(n=640, p=P)
    rect = inputs.dense_full(m=333, n=517, p=P, seed=77).astype(np.uint8)
    lowr = low_rank(rng, 700, 300, 190, P)
    lowr[::7] = 0
    tall = low_rank(rng, 1100, 129, 129, P)
    return {"dense_640": dense, "rect_333x517": rect, "lowrank_700x300": lowr.astype(np.uint8),
            "tall_1100x129": tall.astype(np.uint8)}


CASES = _cases()


def _dev_u8(A, pad=0):
    import torch
    m, n = A.shape
    buf = torch.zeros((m, n + pad), dtype=torch.uint8, device="cuda")
    buf[:, :n] = torch.from_numpy(np.ascontiguousarray(A, dtype=np.uint8)).cuda()
    return buf[:, :n]


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("pad", [0, 13])
def test_factor_u8_matches_oracle(cuda_lib, engine, name, pad):
    import torch
    A = CASES[name]
    want = oracle.cup_packed(A, P)
    h = cuda_lib.Handle(engine=engine)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for call in range(3):               # the second and third calls replay a CUDA graph
            dA = _dev_u8(A, pad)
            r, prof, ipiv = h.factor(dA, P, stream=stream)
            stream.synchronize()
            assert r == want["rank"], (call, r, want["rank"])
            assert np.array_equal(prof[:r].cpu().numpy(), want["profile"])
            assert np.array_equal(ipiv[:r].cpu().numpy(), want["ipiv"])
            assert np.array_equal(dA.cpu().numpy(), want["packed"].astype(np.uint8)), f"call {call}"
    h.close()


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("name", ["dense_640", "lowrank_700x300"])
def test_factor_host_u8(cuda_lib, pinned, name):
    import torch
    A = CASES[name]
    want = oracle.cup_packed(A, P)
    h = cuda_lib.Handle(engine=cuda_lib.ENGINE_TENSOR)
    stream = torch.cuda.Stream()
    for call in range(2):
        hA = torch.from_numpy(np.ascontiguousarray(A, dtype=np.uint8).copy())
        if pinned:
            hA = hA.pin_memory()
        dA = torch.empty(A.shape, dtype=torch.uint8, device="cuda")
        out = torch.empty_like(hA)
        r, prof, ipiv = h.factor_host(hA, dA, P, out=out, stream=stream)
        assert r == want["rank"]
        assert np.array_equal(prof[:r].cpu().numpy(), want["profile"])
        assert np.array_equal(out.numpy(), want["packed"].astype(np.uint8)), f"call {call}"
        assert np.array_equal(dA.cpu().numpy(), want["packed"].astype(np.uint8))
        assert np.array_equal(hA.numpy(), A)             # input untouched when out is another buffer
    h.close()


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("n", [1, 64, 300, 517])
def test_det_inverse_u8(cuda_lib, engine, n):
    A = inputs.dense_full(n=n, p=P, seed=900 + n).astype(np.uint8)
    h = cuda_lib.Handle(engine=engine)
    assert h.det(_dev_u8(A), P) == oracle.det(A, P)
    inv = oracle.inverse(A, P)
    dA = _dev_u8(A, pad=3)
    ok = h.inverse(dA, P)
    assert ok == (inv is not None)
    if inv is not None:
        assert np.array_equal(dA.cpu().numpy(), inv.astype(np.uint8))
    h.close()


def test_inverse_u8_singular_leaves_factors(cuda_lib):
    rng = np.random.default_rng(3)
    A = low_rank(rng, 200, 200, 150, P).astype(np.uint8)
    want = oracle.cup_packed(A, P)
    h = cuda_lib.Handle()
    dA = _dev_u8(A)
    assert h.inverse(dA, P) is False
    assert np.array_equal(dA.cpu().numpy(), want["packed"].astype(np.uint8))
    assert h.det(_dev_u8(A), P) == 0
    h.close()


def test_u8_rejects_large_primes(cuda_lib):
    import torch
    h = cuda_lib.Handle()
    dA = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
    with pytest.raises(cuda_lib.CupError):
        h.factor(dA, 257)
    h.close()
