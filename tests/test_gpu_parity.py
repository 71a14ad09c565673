"""GPU parity: every step of the path through the C-ABI against the CPU oracle
on the same seeded inputs (sizes that span several 32-row slices and end in a
ragged slice).

Bars:
  * residual (Dot2, u_r ~ u^2), A v in u_p, x0 = M b in u_f, the bucketed SpMV,
    bucket ids, ||M||_inf and the stored bucket values: bit-exact (both sides
    run the same sequence of correctly rounded operations per row);
  * SPAI columns: relative 2-norm error per row of M <= max(1e-5, LS bound);
  * GMRES with a fixed number of steps: fp32 1e-4, fp64 1e-10 relative;
  * GMRES-IR solutions (u = fp64): within 1e-12 relative of the oracle's, and
    forward error <= 1e-10.
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import dev, gpu_bucket, gpu_build, host, lib, oracle_M, small_workloads, spai_tolerance

pytestmark = pytest.mark.gpu

WLS = small_workloads()
IDS = [f"{w['name']}-{w['A'].n}" for w in WLS]
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def B():
    return lib()


@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_residual_dd_bitexact(B, wl):
    A = wl["A"]
    rng = np.random.default_rng(3)
    x = wl["x_true"] + rng.normal(0, 1e-9, A.n)
    Ah = B.matrix_create(B.DeviceCSR.from_host(A))
    r = torch.empty(A.n, dtype=torch.float64, device="cuda")
    B.residual(Ah, dev(x), dev(wl["b"]), r)
    assert np.array_equal(host(r), O.residual_dd(A, x, wl["b"]))


@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_spmv_up_bitexact(B, wl):
    A = wl["A"]
    v = np.random.default_rng(4).uniform(-1, 1, A.n).astype(np.float32)
    Ah = B.matrix_create(B.DeviceCSR.from_host(A))
    w = torch.empty(A.n, dtype=torch.float32, device="cuda")
    B.spmv_up(Ah, dev(v), w)
    ref = O.spmv_prec(A.row_ptr, A.col, A.val, "fp32", v.astype(np.float64))
    assert np.array_equal(host(w).astype(np.float64), ref)


def _spai_tolerance(kappa, resid):
    return spai_tolerance(kappa, resid, U32)


@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_spai_matches_oracle(B, wl):
    A, P = wl["A"], wl["pattern"]
    g = gpu_build(B, wl)
    assert g["info"]["n_rank_deficient"] == 0 and g["info"]["status"] == 0
    assert np.array_equal(g["row_ptr"], P.row_ptr) and np.array_equal(g["col"], P.col)
    ref = O.spai(A, P, wl["spai_eps"])
    tol = _spai_tolerance(ref["kappa"], ref["resid"])
    worst = 0.0
    for k in range(A.n):
        a, b = P.row_ptr[k], P.row_ptr[k + 1]
        e = np.linalg.norm(g["val"][a:b] - ref["mval"][a:b]) / np.linalg.norm(ref["mval"][a:b])
        worst = max(worst, e / tol[k])
        assert e <= tol[k], (k, e, tol[k])
    # the column residuals agree, and the Alg 2.1 test flags the same columns
    # except where ||s|| sits within rounding of spai_eps
    assert np.allclose(g["resid"], ref["resid"], rtol=1e-4, atol=1e-6)
    clear = np.abs(ref["resid"] - wl["spai_eps"]) > 1e-4
    assert np.array_equal((g["resid"] <= wl["spai_eps"])[clear], (ref["conv"] == 1)[clear])
    assert g["info"]["n_converged"] == int((g["resid"] <= wl["spai_eps"]).sum())
    print(f"{wl['name']}: worst SPAI error / tolerance = {worst:.3f}")


EPS = [2.0 ** -37, 2.0 ** -24, 2.0 ** -16, 2.0 ** -10]


@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_buckets_bitexact(B, wl):
    P = wl["pattern"]
    M, muf = oracle_M(B, wl)
    plists = [wl["precs"], wl["precs"] + ["drop"], ["fp64"], ["fp32", "bf16", "e4m3"]]
    for precs in plists:
        for eps in EPS:
            b = gpu_bucket(B, M, P.nnz, eps, precs)
            ref = O.bucket_ids(P.row_ptr, muf, eps, precs)
            assert b["info"]["norm_inf"] == ref["norm"]
            assert np.array_equal(b["ids"], ref["ids"]), (precs, eps)
            assert b["info"]["nnz_k"] == ref["nnz_k"].tolist()
            assert b["info"]["thresholds"][1:] == ref["thr"][1:].tolist()
            stored, _, _ = O.bucket_store(P.row_ptr, P.col, muf, ref["ids"], precs)
            assert np.array_equal(b["stored"], stored), (precs, eps)
            assert abs(b["info"]["storage_pct"] - O.storage_pct(ref["nnz_k"], precs, 0)) < 1e-9


@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_bucketed_spmv_bitexact(B, wl):
    P = wl["pattern"]
    M, muf = oracle_M(B, wl)
    rng = np.random.default_rng(5)
    x64 = rng.uniform(-1, 1, P.n)
    x32 = rng.uniform(-1, 1, P.n).astype(np.float32)
    for precs in [wl["precs"], wl["precs"] + ["drop"], ["fp64", "fp32", "fp16", "bf16", "e4m3"]]:
        for eps in EPS:
            b = gpu_bucket(B, M, P.nnz, eps, precs)
            ref = O.bucket_ids(P.row_ptr, muf, eps, precs)
            stored, _, _ = O.bucket_store(P.row_ptr, P.col, muf, ref["ids"], precs)
            for xin, ydt in [(x64, torch.float64), (x32, torch.float32), (x64, torch.float32)]:
                y = torch.empty(P.n, dtype=ydt, device="cuda")
                B.apply(b["BM"], dev(xin), y)
                yr = O.bspmv(P.row_ptr, P.col, stored, ref["ids"], precs, xin.astype(np.float64))
                if ydt == torch.float32:
                    yr = yr.astype(np.float32).astype(np.float64)
                yg = host(y).astype(np.float64)
                # stated bar: 2e-6 relative in the infinity norm; observed: bit-exact
                assert np.abs(yg - yr).max() <= 2e-6 * np.abs(yr).max()
                assert np.array_equal(yg, yr), (precs, eps, ydt)


@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_x0_apply_uf_bitexact(B, wl):
    P = wl["pattern"]
    M, muf = oracle_M(B, wl)
    y = torch.empty(P.n, dtype=torch.float64, device="cuda")
    B.apply_uf(M, dev(wl["b"]), y)
    ref = O.spmv_prec(P.row_ptr, P.col, muf, "fp32", wl["b"])
    assert np.array_equal(host(y), ref)


@pytest.mark.parametrize("ug,tol", [("fp32", 1e-4), ("fp64", 1e-10)])
@pytest.mark.parametrize("wl", WLS[:4], ids=IDS[:4])
def test_gmres_fixed_steps_matches_oracle(B, wl, ug, tol):
    A, P = wl["A"], wl["pattern"]
    M, muf = oracle_M(B, wl)
    precs = wl["precs"]
    eps = 2.0 ** -16
    b = gpu_bucket(B, M, P.nnz, eps, precs)
    ids = O.bucket_ids(P.row_ptr, muf, eps, precs)["ids"]
    stored, _, _ = O.bucket_store(P.row_ptr, P.col, muf, ids, precs)
    S = O.System(A, P.row_ptr, P.col, stored, ids, precs)
    r = O.residual_dd(A, O.spmv_prec(P.row_ptr, P.col, muf, "fp32", wl["b"]), wl["b"])
    k = 8
    d_ref, it_ref, _ = O.gmres(S, r, ug, ug, 0.0, k)
    Ah = B.matrix_create(B.DeviceCSR.from_host(A))
    d = torch.empty(A.n, dtype=torch.float64, device="cuda")
    info = B.gmres(Ah, b["BM"], dev(r), d, ug, ug, B.opts(tau=0.0, kmax=k))
    assert info["gmres_iters"] == [k] and it_ref == k
    dg = host(d)
    assert np.linalg.norm(dg - d_ref) <= tol * np.linalg.norm(d_ref)


@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_gmres_ir_matches_oracle(B, wl):
    """End to end: SPAI build, bucketing, BSPAI-GMRES-IR, against the oracle's
    own pipeline from the same inputs."""
    A, P = wl["A"], wl["pattern"]
    for eps in [2.0 ** -37, 2.0 ** -16]:
        g = gpu_build(B, wl)
        b = gpu_bucket(B, g["M"], P.nnz, eps, wl["precs"])
        x = torch.empty(A.n, dtype=torch.float64, device="cuda")
        info = B.gmres_ir_solve(g["A"], dev(wl["b"]), b["BM"], g["M"], x, tol=wl["tau"])
        xg = host(x)
        ref = O.solve(wl, bucket_eps=eps)
        xt = wl["x_true"]
        assert info["status"] == 0, info
        fe_g = np.abs(xg - xt).max() / np.abs(xt).max()
        fe_o = np.abs(ref["x"] - xt).max() / np.abs(xt).max()
        assert fe_g <= 1e-10 and fe_o <= 1e-10
        assert np.abs(xg - ref["x"]).max() <= 1e-12 * np.abs(ref["x"]).max()
        assert info["stop_reason"] in (1, 2, 3)
        # same number of refinement steps; GMRES counts within a few iterations.  The
        # first step's count is set by the preconditioner; later steps solve for
        # corrections of 1e-5 .. 1e-13 relative, where the count also moves with the
        # summation order of the u_g dot products, which the paper leaves open (the
        # GPU's tree and the oracle's pairwise order differ; a sequential order moved
        # this workload's late counts by 2)
        assert abs(info["ir_steps"] - ref["steps"]) <= 1
        for i, (a, c) in enumerate(zip(info["gmres_iters"], ref["its"])):
            assert abs(a - c) <= (max(2, 0.1 * c) if i == 0 else max(4, 0.2 * c)), (i, a, c)
