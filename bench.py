#!/usr/bin/env python3
"""Benchmark of the GB300 CUP library.

Workload: CUP decomposition (Algorithm 6) of a dense 8192 x 8192 matrix of
uniform residues over GF(65521), uint32 storage, with the Schur updates on
tcgen05 tensor cores (2 centred 8-bit limbs per residue). One step is one
complete in-place factorisation of that matrix; before every step the
pristine input is restored by a device-to-device copy outside the step's
events (the 256 MiB input is also larger than the 129 MiB L2).

Metric: field operations per second normalised by the paper's leading-term
count 2mnr - (m+n)r^2 + 2/3 r^3 (Sec. 4.2), in Gop/s.

  python bench.py [--gpus N --steps K --warmup W]      # our CUDA path
  python bench.py --impl reference ...                   # the CPU oracle, timed on the host

Under torchrun (N > 1) every rank factors its own replica (one CUP does not
shard: its pivot search is sequential down the rows); the value is the
operations of all ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

METRIC = "CUP GF(p) Gop/s (leading-term normalised)"
UNIT = "Gop/s"


def cup_ops(m: int, n: int, r: int) -> float:
    """2mnr - (m+n) r^2 + 2/3 r^3: field operations of CUP with classical products (Sec. 4.2)."""
    return 2.0 * m * n * r - (m + n) * float(r) * r + 2.0 / 3.0 * float(r) ** 3


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="dense_full",
                    choices=["dense_full", "dense_plain", "rank_deficient", "dense_small_p", "batched"],
                    help="dense_full (default): 8192^2 GF(65521); dense_plain: 512^2 rank 384; "
                         "rank_deficient: 16384x4096 rank 3000 GF(8388593); dense_small_p: 32768^2 GF(251); "
                         "batched: 4096 matrices, 64 primes near 2^30")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--p", type=int, default=None)
    ap.add_argument("--engine", choices=["tensor", "plain"], default="tensor")
    ap.add_argument("--op", choices=list(OPS), default="factor",
                    help="operation timed on the workload: factor (CUP, the headline), ple, det, inverse, rref, "
                         "nullspace; inverse, rref and nullspace need a square nonsingular workload")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-engine comparison")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-sample", type=int, default=4096, help="side of the oracle's sample matrix")
    ap.add_argument("--leaf-rows", type=int, default=None)
    ap.add_argument("--window", type=int, default=None)
    ap.add_argument("--tc-min-k", type=int, default=None)
    ap.add_argument("--schedule", type=int, default=None, choices=[0, 1, 2],
                    help="cup_factor schedule: 1 device-resident replayed as a CUDA graph (default), "
                         "2 device-resident eager, 0 host-driven")
    ap.add_argument("--int-path", type=int, default=None, choices=[0, 1, 2],
                    help="int_det images: 0 cost model, 1 batched launch, 2 one CUP per prime")
    ap.add_argument("--profile", type=int, default=0,
                    help="library timing level during the timed steps (0: none, CUDA-graph replay; "
                         "2: every kernel class)")
    ap.add_argument("--roofline-steps", type=int, default=1,
                    help="extra untimed steps run with per-launch GEMM timing for the roofline object")
    ap.add_argument("--no-schur", action="store_true",
                    help="skip the isolated Schur-update measurement (16384^3 over GF(251))")
    ap.add_argument("--schur-only", action="store_true",
                    help="only the isolated Schur update (and the instruction probes), one JSON line")
    ap.add_argument("--schur-n", type=int, default=16384, help="size of the isolated Schur update")
    ap.add_argument("--no-probes", action="store_true", help="skip the tensor-instruction peak probes")
    ap.add_argument("--kernel-only", action="store_true",
                    help="only warm-up and timed factorisations (for profiler launch lists)")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# distributed helpers (also exercised by CPU tests with the gloo backend)
# ---------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, world: int) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def shard_indices(count: int, world: int, rank: int) -> list:
    """The batched workload's matrices this rank factors: every world-th one, from
    its rank on (round robin, so every rank gets the same mix of sizes and primes)."""
    return list(range(rank, count, world))


def gather_batched(count: int, idx: list, recs: list, world: int) -> list:
    """Host-side gather of the per-matrix results of every rank's shard (recs[i] is
    the result of matrix idx[i]: its rank, determinant and row rank profile) into one
    list indexed by matrix, on every rank. There is no device collective: the factor
    launches never exchange data."""
    parts = [(list(idx), list(recs))]
    if world > 1:
        import torch.distributed as dist
        parts = [None] * world
        dist.all_gather_object(parts, (list(idx), list(recs)))
    out = [None] * count
    for ii, rr in parts:
        for b, rec in zip(ii, rr):
            if out[b] is not None:
                raise RuntimeError(f"matrix {b} factored by two ranks")
            out[b] = rec
    if any(r is None for r in out):
        raise RuntimeError("a matrix of the batch was factored by no rank")
    return out


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        # samples under load: the top half of the clock readings
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(rows), "reasons": reasons}


# ---------------------------------------------------------------------------
# workloads (seeded synthetic inputs of the paper's settings)
# ---------------------------------------------------------------------------
def make_workload(args):
    """Returns (name, list of (matrix, p)) for the chosen workload."""
    from paper_1112_5717_gb300 import inputs
    w = args.workload
    if w == "dense_full":
        n = args.n or (512 if args.op == "int_det" else 8192)
        p = args.p or inputs.P_16
        return f"dense_full {n}x{n} uniform over GF({p})", [(inputs.dense_full(n=n, p=p), p)]
    if w == "dense_plain":
        p = args.p or inputs.P_16
        return f"dense_plain 512x512 rank 384 over GF({p}), rows shuffled", [(inputs.dense_plain(p=p), p)]
    if w == "rank_deficient":
        p = args.p or inputs.P_23
        return (f"rank_deficient 16384x4096 rank 3000 over GF({p}), every 7th row zero, every 5th a combination",
                [(inputs.rank_deficient(p=p), p)])
    if w == "dense_small_p":
        n = args.n or 32768
        p = args.p or inputs.P_8
        A = inputs.dense_small_p(n=n, p=p)
        return f"dense_small_p {n}x{n} uniform over GF({p}) (uint8 input, uint32 in the library)", [(A, p)]
    mats = inputs.batched()
    return "batched 4096 matrices, m, n log-uniform in [64, 1024], 64 primes below 2^30", mats


# ---------------------------------------------------------------------------
# the CPU oracle as baseline (test infrastructure, timed as it stands)
# ---------------------------------------------------------------------------
# Operations and their leading-term operation counts (Table 1, omega = 3): CUP, PLE and
# det cost 2mnr - (m+n) r^2 + 2/3 r^3; the reduced echelon transform (inverse, rref,
# nullspace) of a nonsingular n x n matrix costs 2 n^3.
OPS = ("factor", "ple", "det", "inverse", "rref", "nullspace", "trlum", "inplace_mm", "int_det")
_INT_K = [0]      # primes used by the last int_det call


def op_ops(op: str, m: int, n: int, r: int) -> float:
    if op in ("factor", "ple", "det"):
        return cup_ops(m, n, r)
    if op == "int_det":
        # one CUP per prime image
        return _INT_K[0] * cup_ops(m, n, r)
    if m != n or r != n:
        raise SystemExit(f"--op {op} needs a square nonsingular workload")
    if op == "trlum":
        return 2.0 / 3.0 * float(n) ** 3
    if op == "inplace_mm":
        # CUP + TRMM(Up, Unit) + TRMM(Low) + TRLUM with B = A (n x n): (2/3 + 2 + 2/3) n^3
        return 10.0 / 3.0 * float(n) ** 3
    return 2.0 * float(n) ** 3


def op_metric(op: str) -> str:
    if op == "int_det":
        return "int_det over Z by CUP modulo primes + CRT, Gop/s (Table 1 leading term, summed over the prime images)"
    return METRIC if op == "factor" else f"{op} over GF(p) Gop/s (Table 1 leading term)"


def run_op(h, op: str, A, p: int):
    """One call of the operation through the library; returns the rank."""
    if op == "factor":
        return h.factor(A, p)[0]
    if op == "ple":
        return h.ple(A, p)[0]
    if op == "det":
        h.det(A, p)
        return min(A.shape)
    if op == "inverse":
        h.inverse(A, p)
        return A.shape[0]
    if op == "rref":
        return h.rref(A, p)[0]
    if op == "trlum":
        h.trlum(A, p)
        return A.shape[0]
    if op == "int_det":
        _, r, cert, k = h.int_det(A)
        if not cert:
            raise SystemExit("int_det: the bound was not met")
        _INT_K[0] = k
        return r
    if op == "inplace_mm":
        # B <- A B with B a device copy of A, made inside the call
        B = _op_scratch(A)
        B.copy_(A)
        return h.inplace_mm(A, B, p)
    return h.nullspace(A, p)[0]


_SCRATCH = {}


def _op_scratch(A):
    key = (tuple(A.shape), A.device)
    if key not in _SCRATCH:
        _SCRATCH[key] = A.clone()
    return _SCRATCH[key]


def oracle_op(op: str, A, p: int):
    """The oracle's version of the operation; returns the rank."""
    import oracle
    if op == "factor":
        return oracle.cup(A, p)["rank"]
    if op == "ple":
        return oracle.ple(A, p)["rank"]
    if op == "det":
        oracle.det(A, p)
        return min(A.shape)
    if op == "inverse":
        oracle.inverse(A, p)
        return A.shape[0]
    if op == "rref":
        return oracle.rref(A, p, want_x=True)["rank"]
    if op == "trlum":
        oracle.trlum(A, p)
        return A.shape[0]
    if op == "inplace_mm":
        oracle.inplace_mm(A, A, p)
        return oracle.cup(A, p)["rank"]
    return oracle.nullspace(A, p)["rank"]


def oracle_sample(n: int, p: int, workload: str = "dense_full", op: str = "factor"):
    """Times the oracle on one bounded sample of the workload; returns
    (Gop/s, seconds, threads, description)."""
    import oracle
    from paper_1112_5717_gb300 import inputs
    if workload == "batched":
        mats = inputs.batched(count=64)
        desc = "CUP of the first 64 matrices of the batched workload"
    elif workload == "rank_deficient":
        mats = [(inputs.rank_deficient(m=4 * n, n=n, r=(3 * n) // 4, p=p), p)]
        desc = f"CUP of one {4 * n}x{n} rank-{(3 * n) // 4} matrix of the rank-deficient structure"
    elif workload == "dense_plain":
        mats = [(inputs.dense_plain(p=p), p)]
        desc = "CUP of the 512x512 rank-384 workload itself"
    else:
        mats = [(inputs.dense_full(n=n, p=p, seed=inputs.SEED_BASE + 2), p)]
        desc = f"CUP of one {n}x{n} uniform matrix over GF({p}) (the workload scaled down)"
    if op != "factor":
        desc = desc.replace("CUP", op, 1)
    if op == "int_det":
        # the same per-image work: CUP modulo each of 4 primes near 2^30 of a centred matrix
        import numpy as np
        A = mats[0][0]
        q0 = int(mats[0][1])
        Z = A.astype(np.int64) - q0 // 2
        qs = inputs.primes_below(1 << 30, 4)
        t0 = time.perf_counter()
        for q in qs:
            oracle.det((Z % q).astype(np.uint32), q)
        dt = time.perf_counter() - t0
        ops = len(qs) * cup_ops(A.shape[0], A.shape[1], min(A.shape))
        return (ops / dt / 1e9, dt, oracle.num_threads(),
                f"det modulo 4 primes near 2^30 of one {A.shape[0]}x{A.shape[1]} centred integer matrix")
    t0 = time.perf_counter()
    ops = 0.0
    for A, q in mats:
        rr = oracle_op(op, A, q)
        ops += op_ops(op, A.shape[0], A.shape[1], rr)
    dt = time.perf_counter() - t0
    return ops / dt / 1e9, dt, oracle.num_threads(), desc


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    n = args.cpu_sample
    p = args.p or 65521
    for _ in range(args.warmup):
        oracle_sample(n, p, args.workload, args.op)
    vals, times = [], []
    for _ in range(args.steps):
        v, dt, cores, desc = oracle_sample(n, p, args.workload, args.op)
        vals.append(v)
        times.append(dt)
    value = statistics.median(vals)
    sample = f"{desc}, per step; leading-term ops / wall time"
    out = {"impl": "reference", "metric": op_metric(args.op), "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(times) * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
           "data": "synthetic",
           "config": {"workload": f"{args.workload} (sampled on the host: {sample})", "p": p},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    import paper_1112_5717_gb300 as cup

    world, rank, local = dist_env()
    if args.schur_only:
        torch.cuda.set_device(local)
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        try:
            peaks = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")))
        except (OSError, ValueError):
            peaks = {}
        out = measure_schur(cup, torch.cuda.current_device(), stream, peaks, n=args.schur_n,
                            probes_on=not args.no_probes)
        if rank == 0:
            print(json.dumps({"schur": out}), flush=True)
        return 0
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    engine = cup.ENGINE_TENSOR if args.engine == "tensor" else cup.ENGINE_PLAIN
    wname, mats = make_workload(args)
    batched = args.workload == "batched"
    count_all = len(mats)
    shard = list(range(count_all))
    if batched and world > 1:
        # the batch's matrices are independent problems: each rank factors its share
        shard = shard_indices(count_all, world, rank)
        mats = [mats[i] for i in shard]

    # pristine inputs resident in HBM (and pinned host copies for the end-to-end leg)
    if args.op == "int_det":
        # the integer matrix: the residues centred around zero, int64
        hosts = [torch.from_numpy(np.ascontiguousarray(A, dtype=np.int64) - int(q) // 2).pin_memory()
                 for A, q in mats]
    elif mats[0][0].dtype == np.uint8 and args.op in ("factor", "det", "inverse"):
        # one-byte storage at the boundary (the library widens a working copy itself)
        hosts = [torch.from_numpy(np.ascontiguousarray(A)).pin_memory() for A, _ in mats]
    else:
        hosts = [torch.from_numpy(np.ascontiguousarray(A, dtype=np.uint32).view(np.int32)).pin_memory()
                 for A, _ in mats]
    primes = [int(q) for _, q in mats]
    pristine = [t.to(dev) for t in hosts]
    work = [torch.empty_like(t) for t in pristine]
    opts = {k: v for k, v in (("leaf_rows", args.leaf_rows), ("window", args.window),
                              ("tc_min_k", args.tc_min_k), ("int_path", args.int_path),
                              ("schedule", args.schedule)) if v is not None}
    h = cup.Handle(dev, engine=engine, profile=args.profile, **opts)
    # a stream of our own (calls repeated on it may be replayed as CUDA graphs)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    def restore():
        for w_, p_ in zip(work, pristine):
            w_.copy_(p_)

    if batched and args.op != "factor":
        raise SystemExit("the batched workload times the factorization only")

    def compute():
        if batched:
            ranks, _, _, _ = h.factor_batched(work, primes)
            return ranks
        return run_op(h, args.op, work[0], primes[0])

    def one_step():
        restore()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = compute()
        e1.record(stream)
        return out, e0, e1

    for _ in range(args.warmup):
        out, _, _ = one_step()
    torch.cuda.synchronize()
    if batched:
        ranks_v = out.cpu().numpy().tolist()
    else:
        ranks_v = [out]
    ops = sum(op_ops(args.op, A.shape[0], A.shape[1], rr) for (A, _), rr in zip(mats, ranks_v))
    h.reset_stats()
    clocks = ClockSampler(dev)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        _, e0, e1 = one_step()
        evs.append((e0, e1))
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    st = h.stats()
    # roofline figures from extra steps outside the timed region, with the
    # dominant kernel timed per launch by CUDA events on the library's stream
    rst, rstep_ms = st, sum(step_ms)
    if args.profile == 0 and args.roofline_steps > 0:
        h.set_option(cup.OPT_PROFILE, 1)
        h.reset_stats()
        revs = []
        for _ in range(args.roofline_steps):
            _, e0, e1 = one_step()
            revs.append((e0, e1))
        torch.cuda.synchronize()
        rst = h.stats()
        rstep_ms = sum(a.elapsed_time(b) for a, b in revs)
        h.set_option(cup.OPT_PROFILE, 0)
    gathered = None
    if batched:
        # each rank's per-matrix results (rank, det, row rank profile), gathered on the host
        restore()
        rk, prs, _, dts = h.factor_batched(work, primes, want_det=True)
        torch.cuda.synchronize()
        rk, dts = rk.cpu().numpy().tolist(), dts.cpu().numpy().view(np.uint32).tolist()
        recs = [[rk[i], dts[i] if mats[i][0].shape[0] == mats[i][0].shape[1] else None,
                 prs[i][:rk[i]].cpu().numpy().tolist()] for i in range(len(mats))]
        allrec = gather_batched(count_all, shard, recs, world)
        gathered = {"matrices": len(allrec), "ranks": world, "rank_sum": int(sum(r[0] for r in allrec)),
                    "square_dets": sum(1 for r in allrec if r[1] is not None)}
    ms = statistics.mean(step_ms)
    ms_max = max_over_ranks(ms, world)
    # replicas: every rank did the same work; a sharded batch: each rank its share
    ops_all = sum_over_ranks(ops, world) if batched else ops * world
    value = ops_all / (ms_max * 1e-3) / 1e9
    shape = {"matrices": len(mats)} if batched else {"m": mats[0][0].shape[0], "n": mats[0][0].shape[1],
                                                     "p": primes[0], "rank": ranks_v[0]}
    result = {"metric": op_metric(args.op), "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
              "scaling": "strong" if (batched and world > 1) else "weak",
              "vs_baseline": None, "dtype": "u8" if hosts[0].dtype == torch.uint8 else "u32", "data": "synthetic",
              "config": dict({"workload": wname + (" (one persistent launch)" if batched else
                                                   (f", in-place CUP (Algorithm 6), {args.engine} Schur updates" if args.op == "factor" else
                                                    f", {args.op} through the library (CUP, Algorithms 5 and 7-9 or Sec. 5), "
                                                    f"{args.engine} Schur updates")),
                              "engine": args.engine, "leading_term_ops": ops_all,
                              "limbs": (cup_limbs(primes[0]) if args.op != "int_det" else 4)
                                       if engine == cup.ENGINE_TENSOR else None,
                              "l2": "inputs restored by a device copy before each step; the inputs total "
                                    f"{sum(t.numel() * t.element_size() for t in hosts) / 2**20:.0f} MiB "
                                    "(the L2 holds 129 MiB)",
                              "parallelism": ("sharded batch: every rank factors every world-th matrix"
                                              if batched else "replicas") if world > 1 else "single",
                              "options": opts,
                              "step_ms_min": min(step_ms), "step_ms_max": max(step_ms)}, **shape),
              "gpu_launches": int(st["launches"]),
              "clocks": clk}
    if gathered:
        result["batch_gather"] = gathered

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    if rst["tc_launches"] and rst["tc_ms"] > 0:
        achieved = rst["tc_limb_flops"] / (rst["tc_ms"] * 1e-3) / 1e12
        peak = peaks.get("bf16_tflops")
        src = "measured burst bf16 (MEASURED_PEAKS.json)"
        if peak is None:
            peak, src = 1900.0, "fallback 1.9 PFLOP/s bf16"
        tsteps = args.roofline_steps if args.profile == 0 else args.steps
        traffic, tnote = captured_traffic(wkey(args, opts, engine == cup.ENGINE_TENSOR),
                                          rst["tc_launches"] / max(tsteps, 1))
        result["roofline"] = {"bound": "tensor", "kernel": "k_limb_gemm", "achieved": achieved, "peak": peak,
                              "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                              "traffic_unit": "bytes per launch", "traffic_source": tnote,
                              "algorithmic_bytes_per_launch": rst.get("tc_alg_bytes", 0.0) / rst["tc_launches"],
                              "peak_source": src,
                              "per_launch_ms": rst["tc_ms"] / rst["tc_launches"],
                              "launches": rst["tc_launches"],
                              "field_tops": rst["tc_field_flops"] / (rst["tc_ms"] * 1e-3) / 1e12,
                              "share_of_step": rst["tc_ms"] / rstep_ms,
                              "timed_steps": args.roofline_steps if args.profile == 0 else args.steps}
    elif rst["cc_launches"] and rst["cc_ms"] > 0:
        result["roofline"] = {"bound": "alu", "kernel": "k_gemm_sub_cc",
                              "achieved": rst["cc_field_flops"] / (rst["cc_ms"] * 1e-3) / 1e12,
                              "peak": None, "unit": "Tfield-op/s", "frac": None, "traffic": None}
    if world == 1 and not args.no_schur and not args.kernel_only:
        result["schur"] = measure_schur(cup, dev, stream, peaks, n=args.schur_n, probes_on=not args.no_probes)
    result["stats"] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in st.items()}
    if args.profile >= 2:
        result["class_ms_per_step"] = {k: round(v / args.steps, 3) for k, v in h.class_ms().items() if v}

    if args.kernel_only:
        if rank == 0:
            print(json.dumps(result), flush=True)
        return 0

    # end to end through the public API with host buffers
    if not args.no_e2e:
        outs = [torch.empty_like(t).pin_memory() for t in hosts]
        e2e_ms = []
        # untimed calls first: the host-buffer call is captured as a graph on its second call
        e2e_warm = 2 if (args.op == "factor" and not batched) else 1
        for i in range(max(args.steps, 1) + e2e_warm):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if args.op == "factor" and not batched:
                # the library's host-buffer call: row chunks of the input overlap the factorization
                h.factor_host(hosts[0], work[0], primes[0], out=outs[0])
                res_h = None
            else:
                for w_, t in zip(work, hosts):
                    w_.copy_(t, non_blocking=True)
                res = compute()
                for o, w_ in zip(outs, work):
                    o.copy_(w_, non_blocking=True)
                res_h = res.to("cpu", non_blocking=True) if batched else None
            e1.record(stream)
            torch.cuda.synchronize()
            if i >= e2e_warm:
                e2e_ms.append(e0.elapsed_time(e1))
        e_ms = max_over_ranks(statistics.mean(e2e_ms), world)
        nbytes = sum(t.numel() * t.element_size() for t in hosts)
        result["e2e"] = {"value": ops * world / (e_ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": e_ms,
                         "h2d_bytes_per_step": int(nbytes),
                         "d2h_bytes_per_step": int(nbytes + (res_h.numel() * 8 if batched else 0))}

    # the plain CUDA-core INT64 engine on the same workload
    if not args.no_plain and engine == cup.ENGINE_TENSOR and world == 1 and not batched:
        hp = cup.Handle(dev, engine=cup.ENGINE_PLAIN, **opts)
        restore()
        run_op(hp, args.op, work[0], primes[0])
        pm = []
        for _ in range(2):
            restore()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run_op(hp, args.op, work[0], primes[0])
            e1.record(stream)
            torch.cuda.synchronize()
            pm.append(e0.elapsed_time(e1))
        pms = statistics.mean(pm)
        result["plain"] = {"value": ops / (pms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": pms,
                           "tensor_over_plain": pms / ms}
        hp.close()

    if rank == 0 and world == 1 and not args.no_cpu:
        v, dt, cores, desc = oracle_sample(args.cpu_sample, primes[0] if not batched else 0, args.workload,
                                           args.op)
        result["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                  "sample": f"{desc} ({dt:.1f} s), leading-term ops / wall time"}
    if rank == 0:
        print(json.dumps(result), flush=True)
    h.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# DRAM traffic per launch of the tensor-core update, from an ncu capture, keyed by
# workload and valid only for the kernel source it was taken with.
TRAFFIC_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "roofline_traffic.json")
TC_SOURCE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1112_5717_gb300", "csrc", "cup_tc.cu")


def wkey(args, opts, tensor: bool) -> str:
    """Name of the timed configuration in the traffic file (default options only)."""
    if opts or not tensor or args.p:
        return ""
    return f"{args.workload}:{args.n or 'default'}:{args.op}"


def captured_traffic(key: str, launches_per_step=None):
    """(bytes per launch, source) from the traffic file when it holds a capture of this
    configuration taken with the current tensor-kernel source and the same number of
    tensor-kernel launches per step; else (None, why)."""
    import hashlib
    try:
        data = json.load(open(TRAFFIC_FILE))
    except (OSError, ValueError):
        return None, "no ncu capture recorded"
    rec = data.get(key) if key else None
    if not rec:
        return None, "no ncu capture of this configuration"
    sha = hashlib.sha256(open(TC_SOURCE, "rb").read()).hexdigest()
    if rec.get("source_sha256") != sha:
        return None, "stale: the tensor kernel changed since its ncu capture"
    if launches_per_step and rec.get("launches") and round(launches_per_step) != rec["launches"]:
        return None, "stale: the step's tensor-kernel launches changed since its ncu capture"
    return rec["bytes_per_launch"], rec.get("capture", "ncu")


def measure_schur(cup, dev, stream, peaks, n: int = 16384, p: int = 251, warm: int = 2, steps: int = 3,
                  probes_on: bool = True):
    """The Schur update C <- C - A B mod p alone at n^3 over GF(251) (one centred
    8-bit limb, the 32768^2 workload's update shape at n >= 16384), tensor engine:
    CUDA events on the library's stream around the tensor-core kernel only (the
    limb split is a separate launch, timed with the call)."""
    import torch
    g = torch.Generator(device=f"cuda:{dev}")
    g.manual_seed(16384)
    A = torch.randint(0, p, (n, n), dtype=torch.int32, device=dev, generator=g)
    B = torch.randint(0, p, (n, n), dtype=torch.int32, device=dev, generator=g)
    C0 = torch.randint(0, p, (n, n), dtype=torch.int32, device=dev, generator=g)
    C = torch.empty_like(C0)
    hs = cup.Handle(dev, engine=cup.ENGINE_TENSOR, profile=1)
    calls = []
    for i in range(warm + steps):
        C.copy_(C0)
        if i == warm:
            hs.reset_stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hs.mm_sub(C, A, B, p, engine=cup.ENGINE_TENSOR)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= warm:
            calls.append(e0.elapsed_time(e1))
    st = hs.stats()
    hs.close()
    probes = {}
    for kind, name in (((0, "int8_mma_sync_tops"), (1, "bf16_mma_sync_tflops"), (2, "tcgen05_f16_tflops"))
                       if probes_on else ()):
        try:
            probes[name] = cup.probe_tensor_peak(kind, device=dev)
        except Exception as e:                     # reported, not fatal to the benchmark line
            probes[name] = f"failed: {e}"
    L = cup_limbs(p)
    kms = st["tc_ms"] / max(st["tc_launches"], 1)
    limb = 2.0 * L * L * n * n * n
    peak = peaks.get("bf16_tflops") or 1900.0
    achieved = limb / (kms * 1e-3) / 1e12
    return {"m": n, "n": n, "k": n, "p": p, "limbs": L,
            "instruction": "tcgen05.mma.cta_group::1.kind::f16 (bf16 digits, fp32 accumulate in TMEM)",
            "kernel_ms": kms, "call_ms": statistics.mean(calls), "achieved": achieved, "unit": "TFLOP/s",
            "peak": peak, "peak_source": "measured burst bf16 (MEASURED_PEAKS.json)" if peaks.get("bf16_tflops")
            else "fallback 1.9 PFLOP/s bf16", "frac": achieved / peak,
            "field_tops": 2.0 * n * n * n / (kms * 1e-3) / 1e12,
            "instruction_peaks": probes,
            "instruction_peaks_how": "cup_probe_tensor_peak: back-to-back instructions on resident operands, every SM"}


def cup_limbs(p: int) -> int:
    return 1 if p < 2 ** 8 else 2 if p < 2 ** 16 else 3 if p < 2 ** 24 else 4


def main(argv=None):
    args = parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    if args.impl == "reference":
        return run_reference(args)
    import paper_1112_5717_gb300.build as b
    b.build()
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
