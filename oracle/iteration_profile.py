"""Runs the oracle's complete BSPAI-GMRES-IR on a named workload and records
its GMRES iteration profile and timings.

TEST INFRASTRUCTURE ONLY: calls nothing but the oracle.  The benchmark's CPU
baseline (which times a bounded sample of the oracle's phases) reads the
recorded per-step iteration counts to scale that sample to one full solve.

    python oracle/iteration_profile.py convdiff3d 128 0.0009765625
writes oracle/iteration_profile_<workload>_<grid>.json
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2307_03914_gb300 import workloads as W  # noqa: E402


def main(name="convdiff3d", grid=128, bucket_eps=2.0 ** -10, kmax=400):
    wl = W.workload(name, grid=int(grid))
    t0 = time.time()
    out = O.solve(wl, bucket_eps=float(bucket_eps), kmax=int(kmax))
    dt = time.time() - t0
    xt = wl["x_true"]
    fe = float(np.abs(out["x"] - xt).max() / np.abs(xt).max())
    rec = dict(workload=name, grid=int(grid), n=wl["A"].n, bucket_eps=float(bucket_eps),
               precs=wl["precs"], tau=wl["tau"], kmax=int(kmax), its=[int(k) for k in out["its"]],
               steps=int(out["steps"]), stop=int(out["stop"]), nbe=out["nbe"], fwd_err=fe,
               nnz_k=[int(v) for v in out["buckets"]["nnz_k"]], seconds=dt, threads=O.get_threads())
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        f"iteration_profile_{name}_{int(grid)}.json")
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    main(*sys.argv[1:])
