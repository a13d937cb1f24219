"""The tuning table (cup_set_tuning): rules select schedule options per call, options set
explicitly take precedence, malformed tables are refused, and the factors stay
exactly the oracle's whichever options a rule picks."""
import json

import numpy as np
import pytest

import oracle
from paper_1112_5717_gb300 import inputs

pytestmark = pytest.mark.gpu


def _launches(cup, h, A, p):
    import torch
    d = torch.from_numpy(A.view(np.int32).copy()).cuda()
    h.reset_stats()
    r, prof, ipiv = h.factor(d, p)
    torch.cuda.synchronize()
    return h.stats()["launches"], d.cpu().numpy().view(np.uint32), r


def test_rules_select_options_and_keep_results(cuda_lib):
    p = inputs.P_16
    A = inputs.dense_full(n=600, p=p)
    want = oracle.cup_packed(A, p)
    ref = cuda_lib.Handle(tuning=False, schedule=2, leaf_rows=32)
    n_ref, out_ref, _ = _launches(cuda_lib, ref, A, p)
    table = {"entries": [
        {"limbs": 3, "leaf_rows": 16, "window": 40, "tc_min_k": 8},        # another limb count: skipped
        {"limbs": 2, "tall": 1, "leaf_rows": 8},                          # tall calls only: skipped
        {"limbs": 2, "min_lo": 0, "min_hi": 1000, "leaf_rows": 32, "window": 70, "tc_min_k": 64,
         "ms": 1.5, "workload": "note", "candidates": [[32, 70, 64, 1.5]]},
        {"leaf_rows": 64}]}
    h = cuda_lib.Handle(tuning=json.dumps(table), schedule=2)
    n_tab, out_tab, r = _launches(cuda_lib, h, A, p)
    assert n_tab == n_ref                   # the same leaf size as leaf_rows=32 set directly
    assert r == want["rank"]
    assert np.array_equal(out_tab, want["packed"]) and np.array_equal(out_ref, want["packed"])
    # an option set with cup_set_option wins over the table
    h.set_option(cuda_lib.OPT_LEAF_ROWS, 64)
    n_user, out_user, _ = _launches(cuda_lib, h, A, p)
    assert n_user < n_tab
    assert np.array_equal(out_user, want["packed"])
    h.close()
    ref.close()


def test_malformed_tables_are_refused(cuda_lib):
    h = cuda_lib.Handle(tuning=False)
    for bad in ['{"entries": [{"leaf_rows": }]}', '{"rules": []}', '{"entries": [{"leaf_rows" 3}]}',
                '{"entries": [1, 2]}']:
        assert h.lib.cup_set_tuning(h.h, bad.encode()) == -1, bad
    assert h.lib.cup_set_tuning(h.h, b'{"entries": []}') == 0
    assert h.lib.cup_set_tuning(h.h, None) == 0
    h.close()


def test_committed_table_loads(cuda_lib):
    """Every handle loads the table tune.py wrote (when present); the parity tests run under it."""
    import os
    if not os.path.exists(cuda_lib.TUNING_PATH):
        pytest.skip("no tuning table committed")
    h = cuda_lib.Handle()
    text = open(cuda_lib.TUNING_PATH).read()
    assert h.lib.cup_set_tuning(h.h, text.encode()) == 0
    h.close()
