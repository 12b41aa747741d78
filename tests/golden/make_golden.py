"""Writes the stored expected values of the full-size ADMM parity tests (tests/golden/*.json).

Every value here comes from the FP64 oracle (``oracle/``) run on the seeded synthetic inputs
of ``paper_1407_1785_gb300.synth``; nothing is computed by the CUDA library.  The benchmark
workloads are too large for the oracle to run inside a GPU test (minutes to an hour of CPU
time each), so this script runs them once and stores, per output tensor:

  * its relative recovery error against the ground truth, ||X - X_true||_F / ||X_true||_F,
  * its Frobenius norm,
  * the values at a seeded sample of entries (``synth.sample_indices``),

which the GPU tests compare with the library's result of the same solve.

The solves follow the ADMM loops of Sec. 4 (completion: eq. proj, eq. shrink, dual ascent)
and Sec. 5 (tensor RPCA: eq. low_rank, eq. sparse, eq. dual) with rho0 = 1e-2, mu = 1.1,
rho_max = 1e10 and tau = 1/rho on the unnormalised Fourier slices, as the oracle implements
them.

Usage:  python tests/golden/make_golden.py [--only video|rpca|color|batch] [--threads T]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1407_1785_gb300 import synth  # noqa: E402

SAMPLES = 1024
BATCH_SAMPLES = 64
SCHEDULE = dict(rho0=1e-2, mu=1.1, rho_max=1e10)


def _flat(x):
    return np.asfortranarray(x).ravel(order="F")


def _summary(X, truth, k):
    idx = synth.sample_indices(X.size, k)
    out = {"norm": float(np.linalg.norm(X)), "sample_idx": [int(i) for i in idx],
           "sample": [float("%.10g" % v) for v in _flat(X)[idx]]}
    if truth is not None:
        out["rse"] = float(np.linalg.norm(X - truth) / np.linalg.norm(truth))
    return out


def _write(name, obj):
    path = os.path.join(HERE, name + ".json")
    with open(path, "w") as f:
        json.dump(obj, f, indent=0, separators=(",", ":"))
        f.write("\n")
    print(f"wrote {path}", flush=True)


def _header(what, cite, iters, dims):
    return {"what": what, "cite": cite, "generator": "tests/golden/make_golden.py (FP64 oracle)",
            "seed": 1, "iters": iters, "dims": [int(d) for d in dims], **SCHEDULE}


def golden_video():
    X, om = synth.workload_video_completion(seed=1)
    iters = 150
    t0 = time.time()
    Xo, _ = oracle.tnn_complete(X * om, om, iters)
    obj = _header("grayscale video completion 144x176x100, 20% observed",
                  "Sec. 4 ADMM: eq. proj, eq. shrink, dual ascent", iters, X.shape)
    obj["X"] = _summary(Xo, X, SAMPLES)
    obj["oracle_seconds"] = time.time() - t0
    _write("video_completion_144x176x100", obj)


def golden_rpca():
    M, L0, S0, sup, lam = synth.workload_rpca(seed=1)
    iters = 200
    t0 = time.time()
    L, S = oracle.trpca(M, lam, iters)
    obj = _header("tensor RPCA 240x320x60, tubal rank 10, 10% entrywise corruption",
                  "Sec. 5 ADMM: eq. low_rank, eq. sparse, eq. dual", iters, M.shape)
    obj["lambda"] = lam
    obj["L"] = _summary(L, L0, SAMPLES)
    obj["S"] = _summary(S, S0, SAMPLES)
    obj["oracle_seconds"] = time.time() - t0
    _write("rpca_240x320x60", obj)


def golden_color():
    X, om = synth.workload_color_video(seed=1)
    iters = 150
    t0 = time.time()
    Xo, _ = oracle.tnn_complete(X * om, om, iters)
    obj = _header("colour video completion 288x352x3x60, 15% observed",
                  "Sec. 4 ADMM: eq. proj, eq. shrink, dual ascent; DFT along modes 3 and 4 "
                  "(Algorithm 1)", iters, X.shape)
    obj["X"] = _summary(Xo, X, SAMPLES)
    obj["oracle_seconds"] = time.time() - t0
    _write("color_video_completion_288x352x3x60", obj)


def golden_batch():
    items = synth.workload_batch(seed=1)
    iters = 100
    t0 = time.time()
    out = []
    for b, it in enumerate(items):
        M = it["M"].astype(np.float64)
        if it["kind"] == "complete":
            Xo, _ = oracle.tnn_complete(M, it["omega"], iters)
            out.append({"kind": "complete", "dims": list(it["dims"]),
                        "X": _summary(Xo, it["truth"], BATCH_SAMPLES)})
        else:
            L, S = oracle.trpca(M, it["lam"], iters)
            out.append({"kind": "rpca", "dims": list(it["dims"]), "lambda": it["lam"],
                        "L": _summary(L, it["truth"], BATCH_SAMPLES),
                        "S": _summary(S, None, BATCH_SAMPLES)})
        print(f"batch tensor {b} done ({time.time() - t0:.0f} s)", flush=True)
    obj = _header("64 uneven tensors (n1, n2 in [48, 256], n3 in [8, 64]), half completion / "
                  "half RPCA", "Sec. 4 and Sec. 5 ADMM loops, one tensor at a time", iters,
                  [len(items)])
    obj["tensors"] = out
    obj["oracle_seconds"] = time.time() - t0
    _write("batch_64_uneven", obj)


JOBS = {"video": golden_video, "rpca": golden_rpca, "color": golden_color, "batch": golden_batch}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", choices=sorted(JOBS), action="append")
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args()
    oracle.build()
    if a.threads:
        oracle.set_num_threads(a.threads)
    for name in (a.only or ["video", "rpca", "batch", "color"]):
        JOBS[name]()


if __name__ == "__main__":
    main()
