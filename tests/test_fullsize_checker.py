"""The full-size parity checker (shape of [C\\U] plus Freivalds' test of
A P^T = C U) on the CPU: it accepts the oracle's results and rejects every
planted single-entry error, and a wrong transposition."""
import numpy as np
import pytest

import oracle
from paper_1112_5717_gb300 import inputs
from tests.test_gpu_fullsize import check_cup_at_scale

CASES = {
    "dense_300": lambda: (inputs.dense_full(n=300), inputs.P_16),
    "rank_def_700x256": lambda: (inputs.rank_deficient(m=700, n=256, r=150), inputs.P_23),
    "wide_p2": lambda: (inputs.dense_full(m=90, n=500, p=2), 2),
    "tall_p3": lambda: (inputs.dense_full(m=500, n=90, p=3), 3),
    "zero": lambda: (np.zeros((40, 50), dtype=np.uint32), 65521),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_checker_accepts_oracle_and_rejects_errors(name):
    A, p = CASES[name]()
    d = oracle.cup_packed(A, p)
    check_cup_at_scale(A, d["packed"], d["profile"], d["ipiv"], d["rank"], p)
    rng = np.random.default_rng(len(name))
    for _ in range(12):
        bad = d["packed"].copy()
        i, j = rng.integers(0, A.shape[0]), rng.integers(0, A.shape[1])
        bad[i, j] = (int(bad[i, j]) + 1 + int(rng.integers(0, max(p - 1, 1)))) % p
        with pytest.raises(AssertionError):
            check_cup_at_scale(A, bad, d["profile"], d["ipiv"], d["rank"], p)
    if d["rank"] >= 2 and A.shape[1] > d["ipiv"][0] + 1:
        ip = d["ipiv"].copy()
        ip[0] += 1
        with pytest.raises(AssertionError):
            check_cup_at_scale(A, d["packed"], d["profile"], ip, d["rank"], p)
