"""Autotuner of the CUP schedule options on the GPU it runs on.

For each limb count of the tensor engine (p below 2^8, 2^16, 2^24, 2^31) and each
shape class (square matrices by size, and tall rank-deficient ones with m >= 2n), it
times the in-place factorization (Algorithm 6, the tensor engine, repeated calls
replayed as a CUDA graph, CUDA events on the call's stream) for every combination of

  leaf_rows  rows of a base-case slab          (the recursion's leaf size)
  window     pivot-search window of a slab     (how far a slab looks for pivots)
  tc_min_k   smallest inner dimension sent to the tensor engine

and writes the fastest combination of each class, with every candidate's time, to
tuning.json next to the library, which every Handle loads (cup_set_tuning). The
options only change the schedule, never the result: the factors are the same for
every choice.

  python -m paper_1112_5717_gb300.tune [--quick] [--out PATH]
"""
from __future__ import annotations

import argparse
import datetime
import itertools
import json
import os
import statistics

HERE = os.path.dirname(os.path.abspath(__file__))
PRIMES = {1: 251, 2: 65521, 3: 8388593, 4: 2147483647}
BIG = 1 << 40


def workloads(quick: bool):
    """(name, limbs, tall, min_lo, min_hi, builder) of every class timed."""
    from . import inputs
    out = []
    for L, p in PRIMES.items():
        sizes = [(2048, 0, 4096), (8192, 4096, BIG)] if L != 1 else [(2048, 0, 4096), (8192, 4096, 16384),
                                                                     (32768, 16384, BIG)]
        if quick:
            sizes = [(2048, 0, 4096), (8192, 4096, BIG)]
        for n, lo, hi in sizes:
            out.append((f"dense {n}x{n} uniform over GF({p})", L, 0, lo, hi,
                        lambda n=n, p=p: inputs.dense_full(n=n, p=p)))
        out.append((f"rank-deficient 16384x4096 rank 3000 over GF({p})", L, 1, 0, BIG,
                    lambda p=p: inputs.rank_deficient(p=p)))
    return out


def candidates(quick: bool):
    # leaf rows below 48 lost in every class on the GB300; K below 32 goes to the
    # CUDA-core update unless tc_min_k admits it to the one-launch short-K update
    leaf = [64] if quick else [48, 64]
    window = [64, 96, 128] if quick else [64, 80, 96, 128]
    tc = [32] if quick else [1, 32, 64]
    return list(itertools.product(leaf, window, tc))


def time_config(cup, src, p, leaf, window, tc, warm=2, steps=3):
    import torch
    h = cup.Handle(src.device.index, engine=cup.ENGINE_TENSOR, tuning=False, leaf_rows=leaf, window=window,
                   tc_min_k=tc)
    work = torch.empty_like(src)
    st = torch.cuda.Stream()
    ts = []
    with torch.cuda.stream(st):
        for i in range(warm + steps):
            work.copy_(src)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            h.factor(work, p, stream=st)
            e1.record(st)
            st.synchronize()
            if i >= warm:
                ts.append(e0.elapsed_time(e1))
    h.close()
    return statistics.median(ts)


def main(argv=None):
    import numpy as np
    import torch
    import paper_1112_5717_gb300 as cup

    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--quick", action="store_true", help="fewer sizes and candidates")
    ap.add_argument("--out", default=os.path.join(HERE, "tuning.json"))
    args = ap.parse_args(argv)
    torch.cuda.set_device(0)
    cands = candidates(args.quick)
    entries = []
    for name, L, tall, lo, hi, build in workloads(args.quick):
        A = build()
        p = PRIMES[L]
        src = torch.from_numpy(np.ascontiguousarray(A, dtype=np.uint32).view(np.int32)).cuda()
        times = [(leaf, window, tc, round(time_config(cup, src, p, leaf, window, tc), 4))
                 for leaf, window, tc in cands]
        best = min(times, key=lambda t: t[3])
        default = next((t[3] for t in times if t[:3] == (64, 96, 64)), None)
        entries.append({"limbs": L, "tall": tall, "min_lo": lo, "min_hi": hi, "leaf_rows": best[0],
                        "window": best[1], "tc_min_k": best[2], "ms": best[3], "default_ms": default,
                        "workload": name, "candidates": [list(t) for t in times]})
        print(f"{name}: leaf {best[0]} window {best[1]} tc_min_k {best[2]}: {best[3]:.3f} ms "
              f"(defaults {default} ms)", flush=True)
        del src
    out = {"device": torch.cuda.get_device_name(0), "when": datetime.datetime.now(datetime.timezone.utc).isoformat(),
           "how": "median of 3 CUDA-event timings after 2 warm-up calls (graph replay), tensor engine",
           "candidates": "[leaf_rows, window, tc_min_k, ms]", "entries": entries}
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {args.out}")


if __name__ == "__main__":
    main()
