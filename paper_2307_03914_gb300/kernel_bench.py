"""Standalone timing of the path's memory-bound kernels on a convection-
diffusion workload, for roofline work and for profiler captures.

    python -m paper_2307_03914_gb300.kernel_bench [--grid 128] [--reps 20] [--once]

Builds A, M = SPAI(A) and the bucketed M (buckets fp64/fp32/fp16/e4m3 at
bucket_eps = 2^-10, the GMRES setting of the benchmark) on the GPU, then times
with CUDA events, the L2 flushed (a 256 MiB write) before every repetition:
the bucketed product M w (fp32 in and out, as inside GMRES) and A v in u_p =
fp32, each in the three kernel forms (compile-time formats, shared-memory
staged, generic register), and the Dot2 residual.  Prints one JSON
line per form with the median time and the algorithmic bytes (indices int32,
x read once, y written once).
--once runs every kernel exactly once per form with no warm-up and no
flush: a short, fixed launch sequence for a profiler (kernel order: fixed-
format M w and A v, staged M w and A v, register M w and A v, residual).
--mixes times M w (fp32 in and out, default kernel form) for several bucket
lists of the same M (one fp32 bucket, one fp16 bucket, fp32 + fp16, fp16 +
e4m3) to separate the cost of the formats from the cost of the mix.
--batch NSYS NRHS runs the batched solver once on a batch of NSYS systems
with NRHS right-hand sides (the 512 x 32 workload's size distribution), and
prints its statistics, time, and the GMRES launches' kernel-class event time
and algorithmic GB/s (a short launch sequence for a profiler).
With --schedule BD,MGS_ROWS,Z_ROWS,M_SCHED[,TEAM_ROWS] (repeatable; Z_ROWS -1 =
every pair that fits; TEAM_ROWS > 0: team mode) it solves the batch once per
given schedule instead of autotuning and prints each one's time.
--adaptive EPS ALPHA times the adaptive SPAI build (beta = 8, identity
start) on the grid (median of --reps builds) and prints its statistics; with
--once it builds exactly once (a short launch sequence for a profiler).
--spai-uf times the fixed-pattern and the adaptive (spai_eps 0.3, alpha 3,
beta 8) SPAI builds on the grid with u_f = fp32 and u_f = half (median of
--reps builds each, CUDA events around the whole build call); with --once
every build runs exactly once, no warm-up (launch order: fixed fp32,
adaptive fp32, fixed half, adaptive half).
--mgs times GMRES runs of K = 2, 8, 16, 32, 64 steps (tau = 0) on the same
system and fits the MGS kernel-class time to a K + b P(K), P(K) = sum over the
steps j < K of the j + 2 grid reductions of step j: a is the cost per Arnoldi
step outside the reductions (launch, prologue, epilogue), b the cost of one
reduction pass.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import bspai as B
from . import workloads as W

VBYTES = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2, "e4m3": 1, "drop": 0}


def spai_uf(grid, reps, once=False):
    wl = W.workload("convdiff3d", grid=grid)
    A = B.DeviceCSR.from_host(wl["A"])
    P = B.DeviceCSR.from_host(wl["pattern"], with_values=False)
    out = {"n": wl["A"].n}
    for u_f in ("fp32", "fp16"):
        for kind in ("fixed", "adaptive"):
            def build():
                if kind == "fixed":
                    return B.bspai_build(A, P, wl["spai_eps"], u_f=u_f)
                return B.bspai_build_adaptive(A, 0.3, 3, 8, u_f=u_f)

            if not once:
                M, info = build()  # warm-up
                M.free()
            ts = []
            for _ in range(1 if once else reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                M, info = build()
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
                M.free()
            out[f"{kind}_{u_f}"] = {"ms": float(np.median(ts)), "n_converged": info["n_converged"],
                                    "max_resid": info["max_resid"], "nnz": int(info["nnz"]),
                                    "solves": int(info["total_solves"])}
    print(json.dumps(out))


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--grid", type=int, default=128)
    p.add_argument("--reps", type=int, default=20)
    p.add_argument("--bucket-eps", type=float, default=2.0 ** -10)
    p.add_argument("--once", action="store_true")
    p.add_argument("--mgs", action="store_true")
    p.add_argument("--mixes", action="store_true")
    p.add_argument("--batch", type=int, nargs=2, default=None, metavar=("NSYS", "NRHS"))
    p.add_argument("--adaptive", type=float, nargs=2, default=None, metavar=("EPS", "ALPHA"))
    p.add_argument("--spai-uf", action="store_true")
    p.add_argument("--schedule", action="append", default=None, metavar="BD,MGS_ROWS,Z_ROWS,M_SCHED[,TEAM_ROWS]")
    a = p.parse_args()
    if a.spai_uf:
        return spai_uf(a.grid, a.reps, a.once)
    if a.batch:
        return batch(a.batch[0], a.batch[1], a.schedule)
    if a.adaptive:
        return adaptive(a.grid, a.adaptive[0], int(a.adaptive[1]), 1 if a.once else a.reps)
    wl = W.workload("convdiff3d", grid=a.grid)
    A = B.DeviceCSR.from_host(wl["A"])
    P = B.DeviceCSR.from_host(wl["pattern"], with_values=False)
    Ah = B.matrix_create(A)
    M, _ = B.bspai_build(A, P, wl["spai_eps"])
    BM, bi = B.bspai_bucket(M, a.bucket_eps, wl["precs"])
    n, nnz = wl["A"].n, wl["A"].nnz
    g = torch.Generator(device="cuda").manual_seed(1)
    x = torch.rand(n, device="cuda", dtype=torch.float32, generator=g)
    y = torch.empty(n, device="cuda", dtype=torch.float32)
    xd = torch.rand(n, device="cuda", dtype=torch.float64, generator=g)
    bd = torch.from_numpy(wl["b"]).cuda()
    rd = torch.empty(n, device="cuda", dtype=torch.float64)
    torch.cuda.synchronize()
    e4m3 = "e4m3" in bi["precs"] and bi["nnz_k"][bi["precs"].index("e4m3")] > 0
    m_bytes = sum(c * (VBYTES[q] + 4) for c, q in zip(bi["nnz_k"], bi["precs"]) if q != "drop")
    m_bytes += 4 * n + 4 * n + (4 * n if e4m3 else 0)
    a_bytes = nnz * (4 + 4) + 4 * n + 4 * n
    r_bytes = nnz * (8 + 4) + 3 * 8 * n
    if a.mixes:
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

        def tmed(fn):
            for _ in range(3):
                fn()
            ts = []
            for _ in range(a.reps):
                flush.fill_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return float(np.median(ts))

        for precs, eps in ((["fp32"], 2.0 ** -24), (["fp16"], 2.0 ** -11), (["fp32", "fp16"], 2.0 ** -16),
                           (["fp16", "e4m3"], 2.0 ** -10), (["fp64", "fp32", "fp16", "e4m3"], 2.0 ** -10)):
            BMx, bx = B.bspai_bucket(M, eps, precs)
            mb = sum(c * (VBYTES[q] + 4) for c, q in zip(bx["nnz_k"], bx["precs"]) if q != "drop") + 8 * n
            mb += 4 * n if ("e4m3" in bx["precs"] and bx["nnz_k"][bx["precs"].index("e4m3")] > 0) else 0
            t = tmed(lambda: B.apply(BMx, x, y))
            print(json.dumps({"precs": precs, "eps": eps, "nnz_k": bx["nnz_k"], "us": t * 1e3, "GBs": mb / t / 1e6,
                              "bytes": mb}))
        return
    if a.mgs:
        r = torch.from_numpy(wl["b"]).cuda()
        d = torch.empty(n, device="cuda", dtype=torch.float64)
        ks = (2, 8, 16, 32, 64)
        B.gmres(Ah, BM, r, d, "fp32", "fp32", B.opts(tau=0.0, kmax=8))  # warm-up
        rows = []
        for k in ks:
            B.profile_enable(True)
            B.profile_read(reset=True)
            B.gmres(Ah, BM, r, d, "fp32", "fp32", B.opts(tau=0.0, kmax=k))
            prof = B.profile_read(reset=True)
            B.profile_enable(False)
            rows.append((k, sum(j + 2 for j in range(k)), prof["mgs"][0], prof["bspmv"][0], prof["spmv_A"][0]))
        X = np.array([[k, p] for k, p, *_ in rows], dtype=float)
        coef = np.linalg.lstsq(X, np.array([t for *_, t, _, _ in rows]), rcond=None)[0]
        print(json.dumps({"mgs": [dict(K=k, passes=p, mgs_ms=t, bspmv_ms=bm, spmvA_ms=am) for k, p, t, bm, am in rows],
                          "per_step_us": coef[0] * 1e3, "per_pass_us": coef[1] * 1e3, "n": n}))
        return
    if a.once:
        for form in (B.SPMV_AUTO, B.SPMV_STAGED, B.SPMV_REGISTERS):
            B.set_spmv_form(form)
            B.apply(BM, x, y)
            B.spmv_up(Ah, x, y)
        B.set_spmv_form(B.SPMV_AUTO)
        B.residual(Ah, xd, bd, rd)
        torch.cuda.synchronize()
        print(json.dumps({"once": True, "n": n}))
        return
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timeit(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(a.reps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    for form, name in ((B.SPMV_AUTO, "fixed-format"), (B.SPMV_STAGED, "staged"), (B.SPMV_REGISTERS, "registers")):
        B.set_spmv_form(form)
        tm = timeit(lambda: B.apply(BM, x, y))
        ta = timeit(lambda: B.spmv_up(Ah, x, y))
        print(json.dumps({"form": name, "n": n, "nnz_k": bi["nnz_k"], "precs": bi["precs"],
                          "bspmv_us": tm * 1e3, "bspmv_GBs": m_bytes / tm / 1e6, "bspmv_bytes": m_bytes,
                          "spmvA_us": ta * 1e3, "spmvA_GBs": a_bytes / ta / 1e6, "spmvA_bytes": a_bytes}))
    B.set_spmv_form(B.SPMV_AUTO)
    tr = timeit(lambda: B.residual(Ah, xd, bd, rd))
    print(json.dumps({"kernel": "residual_dd", "n": n, "us": tr * 1e3, "GBs": r_bytes / tr / 1e6, "bytes": r_bytes}))


def adaptive(grid, eps, alpha, reps):
    wl = W.workload("convdiff3d", grid=grid)
    A = B.DeviceCSR.from_host(wl["A"])
    ts = []
    info = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        M, info = B.bspai_build_adaptive(A, eps, alpha, 8)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
        M.free()
    print(json.dumps({"grid": grid, "eps": eps, "alpha": alpha, "ms": float(np.median(ts)), "info": info}))


def batch(nsys, nrhs, schedules=None):
    bw = W.batch_workload(nsys=nsys, nrhs=nrhs)
    A = B.DeviceCSR.from_host(bw["A"])
    P = B.DeviceCSR.from_host(bw["pattern"], with_values=False)
    row_off = torch.from_numpy(bw["row_off"]).cuda()
    Bd = torch.from_numpy(bw["B"].reshape(-1)).cuda()
    X = torch.zeros_like(Bd)
    Ah = B.matrix_create(A)
    M, _ = B.bspai_build(A, P, bw["spai_eps"])
    BM, kinfo = B.bspai_bucket_batched(M, row_off, bw["bucket_eps"], bw["precs"])
    torch.cuda.synchronize()
    for sc in schedules or [None]:
        if sc is not None:
            f = [int(v) for v in sc.split(",")] + [0]
            B.batch_schedule_force(f[0], f[1], f[2], f[3], f[4])
        X.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        B.profile_enable(True)
        B.profile_read(reset=True)
        e0.record()
        try:
            info = B.gmres_ir_solve_batched(Ah, row_off, bw["nrhs"], Bd, BM, M, X, tol=bw["tau"])
        finally:
            B.batch_schedule_force(None)
        e1.record()
        torch.cuda.synchronize()
        prof = B.profile_read(reset=True)
        B.profile_enable(False)
        gm = prof["mgs"][0]
        out = {"batch": [nsys, nrhs], "rows": bw["A"].n, "ms": e0.elapsed_time(e1), "gmres_ms": gm,
               "gmres_GBs": info["gmres_bytes"] / (gm / 1000.0) / 1e9 if gm > 0 else None, **info}
        if sc is None:
            out["tuning"] = B.batch_tune_table()
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
