"""Failure detection on the GPU, without a GPU fault.

Every spin-wait in the tensor-core kernels is bounded: after its limit it records
its site in the handle's device error word and the kernel returns, so the CUDA
context stays usable, and the host maps a set word to CUP_ERR_TIMEOUT.
cup_selftest_wait runs that exact bounded wait on an mbarrier that nothing arrives
at. These tests check the status, the message, that the word is cleared, and that
the handle still computes exact results afterwards.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives(cuda_lib):
    import torch
    h = cuda_lib.Handle(engine=cuda_lib.ENGINE_TENSOR)
    st, msg = h.selftest_wait(limit_us=100000)
    assert st == -5, (st, msg)
    assert "device wait expired (site 99)" in msg
    # the error word was cleared: an ordinary call succeeds and is exact
    p = 65521
    rng = np.random.default_rng(5)
    A = rng.integers(0, p, size=(200, 300))
    B = rng.integers(0, p, size=(300, 150))
    C = rng.integers(0, p, size=(200, 150))
    dC = torch.from_numpy(C.astype(np.int32)).cuda()
    h.mm_sub(dC, torch.from_numpy(A.astype(np.int32)).cuda(), torch.from_numpy(B.astype(np.int32)).cuda(), p)
    torch.cuda.synchronize()
    assert np.array_equal(dC.cpu().numpy().view(np.uint32), oracle.mm_sub(C, A, B, p))
    # a second timeout on the same handle is reported again
    st2, _ = h.selftest_wait(limit_us=1000)
    assert st2 == -5
    h.close()


def test_selftest_rejects_bad_limits(cuda_lib):
    h = cuda_lib.Handle()
    assert h.selftest_wait(limit_us=0)[0] == -1
    assert h.selftest_wait(limit_us=10 ** 8)[0] == -1
    h.close()


def test_kernel_setup_on_every_device(cuda_lib):
    """The raised shared-memory limits are set once per device: a handle on each visible
    device factors exactly (one device here is the common case; the loop covers more)."""
    import torch
    p = 65521
    from paper_1112_5717_gb300 import inputs
    A = inputs.dense_plain(m=192, n=160, r=120, p=p)
    want = oracle.cup_packed(A, p)
    for dev in range(torch.cuda.device_count()):
        with torch.cuda.device(dev):
            h = cuda_lib.Handle(dev, engine=cuda_lib.ENGINE_TENSOR, tc_min_k=1)
            dA = torch.from_numpy(A.view(np.int32).copy()).cuda(dev)
            r, prof, ipiv = h.factor(dA, p)
            torch.cuda.synchronize(dev)
            assert r == want["rank"]
            assert np.array_equal(dA.cpu().numpy().view(np.uint32), want["packed"])
            h.close()
