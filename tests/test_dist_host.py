"""The benchmark's multi-rank host logic on CPU: two gloo ranks on 127.0.0.1.

The factorization itself runs as independent replicas (one per GPU, no
collective on the data path); what the ranks share is the timing protocol:
a barrier around the timed region, the slowest rank's time and the sum of the
ranks' operations. The reference arm runs on rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


_WORKER = r"""
import os, sys, json
sys.path.insert(0, os.environ["CUP_ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%s" % os.environ["MASTER_PORT"],
                        rank=int(os.environ["RANK"]), world_size=int(os.environ["WORLD_SIZE"]))
world, rank, local = bench.dist_env()
bench.barrier(world)
mx = bench.max_over_ranks(1.5 + rank, world)        # ranks hold 1.5 and 2.5
sm = bench.sum_over_ranks(10.0 * (rank + 1), world)  # 10 + 20
bench.barrier(world)
print(json.dumps({"rank": rank, "world": world, "max": mx, "sum": sm}), flush=True)
dist.destroy_process_group()
"""


def _run_ranks(code: str, world: int, extra_env=None, args=()):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUP_ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
        env.update(extra_env or {})
        cmd = [sys.executable, "-c", code] if code else [sys.executable, os.path.join(ROOT, "bench.py"), *args]
        procs.append(subprocess.Popen(cmd, env=env, cwd=ROOT, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = []
    for pr in procs:
        try:
            out, err = pr.communicate(timeout=240)
        except subprocess.TimeoutExpired:
            pr.kill()
            raise
        outs.append((pr.returncode, out, err))
    return outs


def test_timing_reductions_over_two_gloo_ranks():
    outs = _run_ranks(_WORKER, 2)
    for rc, out, err in outs:
        assert rc == 0, err
    got = sorted((json.loads(o.strip().splitlines()[-1]) for _, o, _ in outs), key=lambda d: d["rank"])
    assert [d["world"] for d in got] == [2, 2]
    assert all(d["max"] == 2.5 for d in got)
    assert all(d["sum"] == 30.0 for d in got)


def test_reference_arm_prints_on_rank_zero_only():
    """bench.py --impl reference under two ranks: rank 0 times the oracle on a small
    sample and prints one JSON line; rank 1 exits 0 without output."""
    outs = _run_ranks(None, 2, args=("--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
                                     "--cpu-sample", "96"))
    (rc0, out0, err0), (rc1, out1, err1) = outs
    assert rc0 == 0, err0
    assert rc1 == 0, err1
    assert out1.strip() == ""
    line = json.loads(out0.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_operation_counts_follow_table_1():
    """The benchmark's leading-term counts: CUP's 2mnr - (m+n)r^2 + 2/3 r^3 (the oracle's
    exact count of the recursion, to leading order), and Table 1's constants for the square nonsingular case
    (reduced echelon transform 2 n^3, TRLUM 2/3 n^3, InPlaceMM CUP + 2 TRMM + TRLUM)."""
    import numpy as np

    import bench
    import oracle
    assert bench.cup_ops(8192, 8192, 8192) == pytest.approx(2.0 / 3.0 * 8192 ** 3)
    prof = np.arange(0, 3000, dtype=np.int64)
    assert bench.cup_ops(16384, 4096, 3000) == pytest.approx(oracle.opcount(16384, 4096, prof), rel=1e-3)
    n = 1024
    assert bench.op_ops("factor", n, n, n) == pytest.approx(2.0 / 3.0 * n ** 3)
    assert bench.op_ops("inverse", n, n, n) == pytest.approx(2.0 * n ** 3)
    assert bench.op_ops("rref", n, n, n) == pytest.approx(2.0 * n ** 3)
    assert bench.op_ops("trlum", n, n, n) == pytest.approx(2.0 / 3.0 * n ** 3)
    assert bench.op_ops("inplace_mm", n, n, n) == pytest.approx((2.0 / 3.0 + 2.0 + 2.0 / 3.0) * n ** 3)
    with pytest.raises(SystemExit):
        bench.op_ops("inverse", n, n, n - 1)


_SHARD_WORKER = r"""
import os, sys, json
sys.path.insert(0, os.environ["CUP_ROOT"])
import torch.distributed as dist
import bench
import oracle
from paper_1112_5717_gb300 import inputs
world = int(os.environ["WORLD_SIZE"])
if world > 1:
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%s" % os.environ["MASTER_PORT"],
                            rank=int(os.environ["RANK"]), world_size=world)
world, rank, local = bench.dist_env()
mats = inputs.batched(count=23, lo=8, hi=40, defect=6, seed=inputs.SEED_BASE + 77)
idx = bench.shard_indices(len(mats), world, rank)
recs = []
for b in idx:
    A, q = mats[b]
    d = oracle.cup(A, q)
    det = oracle.det(A, q) if A.shape[0] == A.shape[1] else None
    recs.append([d["rank"], det, d["profile"].tolist()])
out = bench.gather_batched(len(mats), idx, recs, world)
print(json.dumps({"rank": rank, "idx": idx, "all": out}), flush=True)
if world > 1:
    dist.destroy_process_group()
"""


def test_batched_shard_and_gather_match_one_rank():
    """The batched workload split across two gloo ranks (every other matrix, no data-path
    collective; the oracle stands in for each rank's factor launch) and gathered on the
    host gives, on both ranks, exactly the per-matrix results of one rank factoring all."""
    one = _run_ranks(_SHARD_WORKER, 1)
    two = _run_ranks(_SHARD_WORKER, 2)
    for rc, out, err in one + two:
        assert rc == 0, err
    ref = json.loads(one[0][1].strip().splitlines()[-1])
    got = [json.loads(o.strip().splitlines()[-1]) for _, o, _ in two]
    assert ref["idx"] == list(range(23))
    assert sorted(got[0]["idx"] + got[1]["idx"]) == list(range(23))
    assert not set(got[0]["idx"]) & set(got[1]["idx"])
    for g in got:
        assert g["all"] == ref["all"]


def test_gather_rejects_overlaps_and_gaps():
    import bench
    assert bench.gather_batched(3, [0, 1, 2], ["a", "b", "c"], 1) == ["a", "b", "c"]
    with pytest.raises(RuntimeError):
        bench.gather_batched(3, [0, 1], ["a", "b"], 1)
    with pytest.raises(RuntimeError):
        bench.gather_batched(2, [0, 0], ["a", "b"], 1)
    assert bench.shard_indices(10, 3, 1) == [1, 4, 7]
