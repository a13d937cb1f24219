"""Parity of the CUDA path with the CPU oracle, element by element (bit exact).

Each test draws seeded inputs, runs the CUDA entry point through the C ABI
and compares every output with the oracle on the same input.
"""
import numpy as np
import pytest

import oracle
from paper_1112_5717_gb300 import inputs

pytestmark = pytest.mark.gpu

PRIMES = [2, 3, 251, 65521, 8388593, 1073741789, 2147483647]


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("engine", [0])
@pytest.mark.parametrize("M,N,K,p", [(1, 1, 1, 7), (64, 64, 64, 65521), (130, 77, 45, 8388593),
                                     (200, 333, 129, 2147483647), (65, 300, 1000, 1073741789),
                                     (257, 130, 33, 2), (31, 17, 5000, 251)])
def test_mm_sub(cuda_lib, engine, M, N, K, p):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.integers(0, p, size=(M, K))
    B = rng.integers(0, p, size=(K, N))
    C = rng.integers(0, p, size=(M, N))
    want = oracle.mm_sub(C, A, B, p)
    dC = _dev(C)
    cuda_lib.mm_sub(dC, _dev(A), _dev(B), p, engine=engine)
    assert np.array_equal(_host(dC), want)


@pytest.mark.parametrize("m,n,p", [(1, 1, 5), (100, 32, 65521), (333, 97, 8388593),
                                   (64, 300, 2147483647), (1000, 64, 2)])
def test_trsm_ruu(cuda_lib, m, n, p):
    rng = np.random.default_rng(m + n)
    U = rng.integers(0, p, size=(n, n))
    B = rng.integers(0, p, size=(m, n))
    want = oracle.trsm_right_upper_unit(U, B, p)
    dB = _dev(B)
    cuda_lib.trsm_ruu(_dev(U), dB, p)
    assert np.array_equal(_host(dB), want)


@pytest.mark.parametrize("p", [65521, 8388593, 2147483647])
@pytest.mark.parametrize("ld,off", [(100, 0), (101, 1)])
def test_trsm_ruu_strided_triangle(cuda_lib, p, ld, off):
    """The triangle as a view with row stride ld (16-byte aligned rows when ld = 100 and the
    view starts at column 0; unaligned otherwise) and n = 97, so a row ends with a partial
    16-byte piece; every accumulation mode of the leaf (p below 2^16, 2^24, 2^31)."""
    n, m = 97, 150
    rng = np.random.default_rng(ld * 7 + p % 1000)
    U = rng.integers(0, p, size=(n, n))
    B = rng.integers(0, p, size=(m, n))
    want = oracle.trsm_right_upper_unit(U, B, p)
    big = np.zeros((n, ld + off), dtype=np.uint32)
    big[:, off:off + n] = U
    dbig = _dev(big)
    dU = dbig[:, off:off + n]
    dB = _dev(B)
    cuda_lib.trsm_ruu(dU, dB, p)
    assert np.array_equal(_host(dB), want)
    assert np.array_equal(_host(dbig), big)          # the triangle is only read


def test_laswp_cols(cuda_lib):
    import torch
    rng = np.random.default_rng(1)
    m, n = 70, 300
    A = rng.integers(0, 1000, size=(m, n))
    ipiv = np.arange(n)
    for t in range(0, 200):
        ipiv[t] = rng.integers(t, n) if t % 3 else t
    want = oracle.laswp_cols(A, ipiv, 5, 180)
    dA = _dev(A)
    cuda_lib.laswp_cols(dA, torch.from_numpy(ipiv.astype(np.int64)).cuda(), 5, 180)
    assert np.array_equal(_host(dA), want)


def _factor_case(cup, A, p, **opts):
    import torch
    d = oracle.cup_packed(A, p)
    h = cup.Handle(**opts)
    dA = _dev(A)
    r, prof, ipiv = h.factor(dA, p)
    torch.cuda.synchronize()
    assert r == d["rank"]
    assert np.array_equal(prof[:r].cpu().numpy(), d["profile"])
    assert np.array_equal(ipiv[:r].cpu().numpy(), d["ipiv"])
    got = _host(dA)
    if not np.array_equal(got, d["packed"]):
        bad = np.argwhere(got != d["packed"])
        raise AssertionError(f"[C\\U] differs at {len(bad)} entries, first {bad[:5].tolist()}")
    h.close()


P_NARROW_TOP = inputs.primes_below((1 << 32) // 9 + 1, 1)[0]

FACTOR_CASES = {
    "dense_plain_512": lambda: (inputs.dense_plain(), inputs.P_16),
    "dense_full_300": lambda: (inputs.dense_full(n=300), inputs.P_16),
    "rank_def_700x256": lambda: (inputs.rank_deficient(m=700, n=256, r=150), inputs.P_23),
    "wide_90x500_p2": lambda: (inputs.dense_full(m=90, n=500, p=2), 2),
    "tall_500x90_p3": lambda: (inputs.dense_full(m=500, n=90, p=3), 3),
    "zero_40x50": lambda: (np.zeros((40, 50), dtype=np.uint32), 65521),
    "one_row": lambda: (inputs.dense_full(m=1, n=77, p=251), 251),
    "one_col": lambda: (inputs.dense_full(m=77, n=1, p=251), 251),
    "p31": lambda: (inputs.dense_full(n=200, p=2147483647), 2147483647),
    # the largest odd p whose nine-product block-update sums still fit one Montgomery
    # reduction (9 (p-1)^2 < p 2^32), and a p above that bound (wide sums)
    "p_narrow_top": lambda: (inputs.dense_full(n=300, p=P_NARROW_TOP), P_NARROW_TOP),
    "p30": lambda: (inputs.dense_full(n=300, p=1073741789), 1073741789),
}


@pytest.mark.parametrize("name", sorted(FACTOR_CASES))
def test_factor_matches_oracle(cuda_lib, name):
    A, p = FACTOR_CASES[name]()
    _factor_case(cuda_lib, A, p, engine=0)


def _swappy(m, n, p, seed):
    """Low-rank matrix with zeroed leading blocks so that pivots move right."""
    rng = np.random.default_rng(seed)
    r = min(m, n) // 2
    X = rng.integers(0, p, size=(m, r))
    Y = rng.integers(0, p, size=(r, n))
    A = inputs.matmul_mod(X, Y, p)
    A[:, : n // 3] *= (rng.random((m, 1)) < 0.3)
    A[rng.random(m) < 0.2] = 0
    return A.astype(np.uint32)


@pytest.mark.parametrize("leaf,window", [(1, 1), (7, 3), (32, 64), (64, 128), (64, 1), (16, 200 // 2)])
@pytest.mark.parametrize("p", [2, 251, 65521])
def test_factor_leaf_and_window_edges(cuda_lib, leaf, window, p):
    A = _swappy(150, 170, p, seed=leaf * 1000 + window)
    _factor_case(cuda_lib, A, p, engine=0, leaf_rows=leaf, window=window)


@pytest.mark.parametrize("n,p", [(1, 7), (50, 65521), (129, 8388593), (64, 2)])
def test_det(cuda_lib, n, p):
    rng = np.random.default_rng(n)
    for trial in range(3):
        A = rng.integers(0, p, size=(n, n)).astype(np.uint32)
        if trial == 2 and n > 1:
            A[-1] = A[0]
        want = oracle.det(A, p)
        got = cuda_lib.Handle(engine=0).det(_dev(A), p)
        assert got == want


@pytest.mark.parametrize("name", ["dense_plain_512", "rank_def_700x256", "wide_90x500_p2",
                                  "tall_500x90_p3", "p31", "dense_full_300", "p_narrow_top", "p30"])
@pytest.mark.parametrize("tc_min_k", [1, 64])
def test_factor_tensor_engine(cuda_lib, name, tc_min_k):
    A, p = FACTOR_CASES[name]()
    _factor_case(cuda_lib, A, p, engine=1, tc_min_k=tc_min_k)


@pytest.mark.parametrize("schedule", [0, 1, 2])
@pytest.mark.parametrize("name", ["dense_plain_512", "rank_def_700x256", "tall_500x90_p3", "zero_40x50",
                                  "wide_90x500_p2", "p31", "one_row"])
def test_factor_schedules_and_graph_replay(cuda_lib, schedule, name):
    """Host-driven (0), device-resident replayed as a CUDA graph (1) and
    device-resident eager (2): three calls on the same buffer each match the oracle."""
    import torch
    A, p = FACTOR_CASES[name]()
    d = oracle.cup_packed(A, p)
    h = cuda_lib.Handle(engine=1, schedule=schedule)
    dA = _dev(A)
    src = dA.clone()
    stream = torch.cuda.Stream()          # graphs are captured on a stream of our own
    stream.wait_stream(torch.cuda.current_stream())
    for call in range(3):
        with torch.cuda.stream(stream):
            dA.copy_(src)
            r, prof, ipiv = h.factor(dA, p)
        torch.cuda.synchronize()
        assert r == d["rank"], call
        assert np.array_equal(prof[:r].cpu().numpy(), d["profile"]), call
        assert np.array_equal(ipiv[:r].cpu().numpy(), d["ipiv"]), call
        assert np.array_equal(_host(dA), d["packed"]), call
    h.close()


def test_speculation_fallback_is_exact(cuda_lib):
    """A window of one position makes the device-resident schedule take rows as
    dependent that are not; the finish kernel detects it and the call is redone
    host-driven from the saved input."""
    p = 251
    A = _swappy(200, 210, p, seed=77)
    for window in (1, 2, 4):
        _factor_case(cuda_lib, A, p, engine=1, leaf_rows=16, window=window, schedule=1)


@pytest.mark.parametrize("schedule", [0, 1, 2])
@pytest.mark.parametrize("name", ["dense_plain_512", "rank_def_700x256", "tall_500x90_p3", "wide_90x500_p2",
                                  "p31", "one_row", "zero_40x50"])
@pytest.mark.parametrize("pinned,inplace", [(True, False), (True, True), (False, False)])
def test_factor_host_buffers(cuda_lib, schedule, name, pinned, inplace):
    """cup_factor_host: the host input arrives in row chunks that overlap the
    factorization; three calls on the same buffers (replayed as a CUDA graph on a
    stream of our own) each return the oracle's [C\\U] in host memory."""
    import torch
    A, p = FACTOR_CASES[name]()
    d = oracle.cup_packed(A, p)
    h = cuda_lib.Handle(engine=1, schedule=schedule)
    src = torch.from_numpy(np.ascontiguousarray(A, dtype=np.uint32).view(np.int32))
    hA = src.clone().pin_memory() if pinned else src.clone()
    out = hA if inplace else (torch.empty_like(hA).pin_memory() if pinned else torch.empty_like(hA))
    dA = torch.empty(A.shape, dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    for call in range(3):
        if inplace:
            hA.copy_(src)
        with torch.cuda.stream(stream):
            r, prof, ipiv = h.factor_host(hA, dA, p, out=out)
        torch.cuda.synchronize()
        assert r == d["rank"], call
        assert np.array_equal(prof[:r].cpu().numpy(), d["profile"]), call
        assert np.array_equal(ipiv[:r].cpu().numpy(), d["ipiv"]), call
        assert np.array_equal(out.numpy().view(np.uint32).astype(np.int64), d["packed"]), call
        assert np.array_equal(_host(dA), d["packed"]), call
    h.close()


def test_factor_host_speculation_fallback(cuda_lib):
    """A window of one position makes rows be taken as dependent that are not; the
    host-buffer call redoes the factorization from the host input and stays exact."""
    import torch
    p = 251
    A = _swappy(200, 210, p, seed=77)
    d = oracle.cup_packed(A, p)
    h = cuda_lib.Handle(engine=1, leaf_rows=16, window=1)
    hA = torch.from_numpy(np.ascontiguousarray(A, dtype=np.uint32).view(np.int32)).clone().pin_memory()
    dA = torch.empty(A.shape, dtype=torch.int32, device="cuda")
    r, prof, ipiv = h.factor_host(hA, dA, p)
    assert r == d["rank"]
    assert np.array_equal(hA.numpy().view(np.uint32).astype(np.int64), d["packed"])
    h.close()


def _dependent_tail(m, n, r, p, seed):
    """Rank r, the first rows independent and every later row a combination of them: after r
    pivots every slab is made of dependent rows whose residual beyond the window is zero."""
    rng = np.random.default_rng(seed)
    X = rng.integers(0, p, size=(r, r))
    Y = rng.integers(0, p, size=(r, n))
    top = inputs.matmul_mod(X, Y, p)
    Z = rng.integers(0, p, size=(m - r, r))
    return np.vstack([top, inputs.matmul_mod(Z, top, p)]).astype(np.uint32)


def _late_nonzeros(m, n, p, seed):
    """Rows whose first nonzero lies beyond a pivot window (zero in the first 150 columns)
    ahead of ordinary rows, zero rows among them, so that a slab's leading rows move a
    column from beyond the window to its first position."""
    rng = np.random.default_rng(seed)
    A = rng.integers(0, p, size=(m, n))
    lead = rng.random(m) < 0.4
    A[lead, :150] = 0
    A[rng.random(m) < 0.15] = 0
    return A.astype(np.uint32)


def _mixed_panels(m, n, p, seed):
    """Independent rows with dependent ones interleaved (every third row a combination of
    earlier rows, every seventh zero): most 8-row panels hold a row that takes no pivot."""
    rng = np.random.default_rng(seed)
    A = rng.integers(0, p, size=(m, n))
    for i in range(m):
        if i % 7 == 6:
            A[i] = 0
        elif i % 3 == 2:
            c = rng.integers(0, p, size=i)
            A[i] = (c @ A[:i]) % p
    return A.astype(np.uint32)


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("case", ["dependent_tail", "late_nonzeros", "mixed_panels"])
@pytest.mark.parametrize("p", [251, 65521, 8388593])
def test_factor_dependent_rows(cuda_lib, engine, case, p):
    """Slabs made of dependent rows (the scan beyond the window), leading rows whose first
    nonzero is beyond the window, and panels mixing dependent and independent rows (the
    fast path with rows that take no rank position), against the oracle."""
    if case == "dependent_tail":
        A = _dependent_tail(640, 300, 90, p, seed=p % 97)
    elif case == "late_nonzeros":
        A = _late_nonzeros(400, 320, p, seed=p % 89)
    else:
        A = _mixed_panels(300, 260, p, seed=p % 83)
    _factor_case(cuda_lib, A, p, engine=engine, window=64)
