#!/usr/bin/env python3
"""Write the oracle's results at the benchmark workloads' full sizes as SHA-256 digests.

The oracle (``oracle/``, plain iterative elimination on the host) takes minutes per
case at these sizes, too long to rerun inside a GPU test. This script runs it once,
on seeded synthetic inputs from ``paper_1112_5717_gb300.inputs``, and stores a digest
of every output in ``fullsize_digests.json`` next to it. The GPU tests hash the CUDA
path's outputs the same way and compare: equal digests mean equal arrays, element for
element. The digest of each input is stored too, so that a difference in input
generation between machines is reported as such and not as a parity failure.

Only ``oracle/`` and the input generators are called here; nothing comes from the
CUDA path.

Cases (the workloads of the benchmark, the sizes it times):
  dense_full_8192       8192 x 8192 uniform over GF(65521): CUP (packed [C\\U],
                        profile, ipiv, rank), det, inverse
  rank_deficient        16384 x 4096 over GF(8388593), rank 3000, zero and
                        combination rows: CUP, reduced column echelon form R and
                        its transform X
  dense_small_p_8192    8192 x 8192 uniform over GF(251) (one 8-bit limb; the
                        32768^2 workload's structure at a size the oracle finishes):
                        CUP, det, inverse
  batched               the 4096 matrices of the batched workload, each modulo its
                        own prime below 2^30: rank, CUP digest and det (square ones)

  python tests/golden/make_fullsize_digests.py [--only CASE ...]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "fullsize_digests.json")
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1112_5717_gb300 import inputs  # noqa: E402


def digest(*arrays) -> str:
    """SHA-256 of the arrays' values: matrices as little-endian uint32, index
    vectors as little-endian int64, each C-contiguous, concatenated in order."""
    h = hashlib.sha256()
    for a in arrays:
        a = np.asarray(a)
        if a.dtype.kind in "iu" and a.ndim == 1 and a.dtype.itemsize == 8:
            b = np.ascontiguousarray(a, dtype="<i8")
        else:
            b = np.ascontiguousarray(a, dtype="<u4")
        h.update(str(b.shape).encode())
        h.update(b.tobytes())
    return h.hexdigest()


def cup_record(A, p):
    d = oracle.cup_packed(A, p)
    return {"rank": d["rank"], "packed": digest(d["packed"]), "profile": digest(d["profile"]),
            "ipiv": digest(d["ipiv"])}


def case_dense(n, p, seed_name):
    A = inputs.dense_full(n=n, p=p) if seed_name == "dense_full" else inputs.dense_small_p(n=n, p=p)
    rec = {"m": n, "n": n, "p": p, "input": digest(A)}
    t = time.time()
    rec["cup"] = cup_record(A, p)
    rec["det"] = oracle.det(A, p)
    inv = oracle.inverse(A, p)
    rec["inverse"] = None if inv is None else digest(inv)
    rec["oracle_seconds"] = round(time.time() - t, 1)
    return rec


def case_rank_deficient():
    p = inputs.P_23
    A = inputs.rank_deficient(p=p)
    rec = {"m": A.shape[0], "n": A.shape[1], "p": p, "input": digest(A)}
    t = time.time()
    rec["cup"] = cup_record(A, p)
    d = oracle.rref(A, p, want_x=True)
    rec["rref"] = {"rank": d["rank"], "R": digest(d["R"]), "X": digest(d["X"]), "profile": digest(d["profile"])}
    rec["oracle_seconds"] = round(time.time() - t, 1)
    return rec


def case_batched():
    mats = inputs.batched()
    rec = {"count": len(mats), "input": digest(*[A for A, _ in mats]),
           "primes": digest(np.array([q for _, q in mats], dtype=np.int64))}
    t = time.time()
    ranks, cups, dets = [], [], []
    for A, q in mats:
        d = oracle.cup_packed(A, q)
        ranks.append(d["rank"])
        # a short digest per matrix: enough to name the matrices that differ
        cups.append(digest(d["packed"], d["profile"], d["ipiv"])[:16])
        dets.append(oracle.det(A, q) if A.shape[0] == A.shape[1] else None)
    rec["ranks"] = ranks
    rec["cup"] = cups
    rec["det"] = dets
    rec["oracle_seconds"] = round(time.time() - t, 1)
    return rec


CASES = {
    "dense_full_8192": lambda: case_dense(8192, inputs.P_16, "dense_full"),
    "rank_deficient": case_rank_deficient,
    "dense_small_p_8192": lambda: case_dense(8192, inputs.P_8, "dense_small_p"),
    "batched": case_batched,
}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--only", nargs="*", choices=list(CASES), default=list(CASES))
    args = ap.parse_args(argv)
    oracle.build()
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in args.only:
        t = time.time()
        data[name] = CASES[name]()
        data[name]["oracle_threads"] = oracle.num_threads()
        with open(OUT + ".tmp", "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(OUT + ".tmp", OUT)
        print(f"{name}: {time.time() - t:.0f} s", flush=True)


if __name__ == "__main__":
    main()
