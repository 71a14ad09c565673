"""GPU parity of the bucketed A v inside GMRES (Section 3, eq. nbe2 and the
forward-error bound fe2 that it enters): A's own entries bucketed by the
rule of Alg 2.2 with the same precision list and bucket_eps as M's, and A v
inside GMRES taken by the adaptive-precision SpMV (Alg 2.3).

Bars:
  * bucket ids, ||A||_inf and the stored bucket values: bit-exact against the
    oracle's bucketing of A's fp64 values;
  * the bucketed A v: bit-exact against the oracle's Alg 2.3;
  * special cases: one fp64 bucket gives the plain fp64 product of A, one fp32
    bucket the plain fp32 product (both textbook sums in row order), and the
    IR solve with one fp64 bucket is bit-identical to the unbucketed solve
    with A v in u_p = fp64;
  * GMRES with a fixed number of steps: fp32 1e-4, fp64 1e-10 relative;
  * GMRES-IR (u = fp64): within 1e-12 relative of the oracle's solution.
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import dev, gpu_bucket, gpu_build, host, lib, oracle_M, small_workloads

pytestmark = pytest.mark.gpu

WLS = small_workloads()
IDS = [f"{w['name']}-{w['A'].n}" for w in WLS]
EPS = [2.0 ** -37, 2.0 ** -24, 2.0 ** -16, 2.0 ** -10]


@pytest.fixture(scope="module")
def B():
    return lib()


def _bucket_A(B, Ah, nnz, eps, precs):
    BA, info = B.bucket_A(Ah, eps, precs)
    ids, stored = B.bucket_export(BA, nnz)
    return dict(BA=BA, info=info, ids=host(ids), stored=host(stored))


def _oracle_A(A, eps, precs):
    ref = O.bucket_ids(A.row_ptr, A.val, eps, precs)
    stored, _, _ = O.bucket_store(A.row_ptr, A.col, A.val, ref["ids"], precs)
    return ref, stored


@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_bucket_A_bitexact(B, wl):
    A = wl["A"]
    Ah = B.matrix_create(B.DeviceCSR.from_host(A))
    for precs in [wl["precs"], wl["precs"] + ["drop"], ["fp64"], ["fp32", "bf16", "e4m3"],
                  ["fp64", "fp32", "fp16", "bf16", "e4m3"]]:
        for eps in EPS:
            b = _bucket_A(B, Ah, A.nnz, eps, precs)
            ref, stored = _oracle_A(A, eps, precs)
            assert b["info"]["norm_inf"] == ref["norm"]
            assert np.array_equal(b["ids"], ref["ids"]), (precs, eps)
            assert b["info"]["nnz_k"] == ref["nnz_k"].tolist()
            assert b["info"]["thresholds"][1:] == ref["thr"][1:].tolist()
            assert np.array_equal(b["stored"], stored), (precs, eps)
            assert abs(b["info"]["storage_pct"] - O.storage_pct(ref["nnz_k"], precs, 0)) < 1e-9


@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_bucketed_A_spmv_bitexact(B, wl):
    A = wl["A"]
    Ah = B.matrix_create(B.DeviceCSR.from_host(A))
    rng = np.random.default_rng(15)
    x64 = rng.uniform(-1, 1, A.n)
    x32 = rng.uniform(-1, 1, A.n).astype(np.float32)
    for precs in [wl["precs"], wl["precs"] + ["drop"], ["fp64", "fp32", "fp16", "bf16", "e4m3"]]:
        for eps in EPS:
            b = _bucket_A(B, Ah, A.nnz, eps, precs)
            ref, stored = _oracle_A(A, eps, precs)
            for xin, ydt in [(x64, torch.float64), (x32, torch.float32), (x64, torch.float32)]:
                y = torch.empty(A.n, dtype=ydt, device="cuda")
                B.apply(b["BA"], dev(xin), y)
                yr = O.bspmv(A.row_ptr, A.col, stored, ref["ids"], precs, xin.astype(np.float64))
                if ydt == torch.float32:
                    yr = yr.astype(np.float32).astype(np.float64)
                assert np.array_equal(host(y).astype(np.float64), yr), (precs, eps, ydt)


@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_single_bucket_A_is_plain_product(B, wl):
    """q = 1: every entry in one bucket, so Alg 2.3 is the ordinary product of
    A rounded to that format, summed in row order (no scaling for fp64/fp32)."""
    A = wl["A"]
    Ah = B.matrix_create(B.DeviceCSR.from_host(A))
    x = np.random.default_rng(16).uniform(-1, 1, A.n)
    y = torch.empty(A.n, dtype=torch.float64, device="cuda")
    b = _bucket_A(B, Ah, A.nnz, 2.0 ** -24, ["fp64"])
    assert b["info"]["nnz_k"] == [A.nnz]
    B.apply(b["BA"], dev(x), y)
    assert np.array_equal(host(y), O.spmv_prec(A.row_ptr, A.col, A.val, "fp64", x))
    x32 = x.astype(np.float32)
    b = _bucket_A(B, Ah, A.nnz, 2.0 ** -24, ["fp32"])
    B.apply(b["BA"], dev(x32), y)
    assert np.array_equal(host(y), O.spmv_prec(A.row_ptr, A.col, A.val, "fp32", x32.astype(np.float64)))


@pytest.mark.parametrize("ug,tol", [("fp32", 1e-4), ("fp64", 1e-10)])
@pytest.mark.parametrize("wl", WLS[:4], ids=IDS[:4])
def test_gmres_b_fixed_steps_matches_oracle(B, wl, ug, tol):
    A, P = wl["A"], wl["pattern"]
    M, muf = oracle_M(B, wl)
    precs = wl["precs"]
    eps = 2.0 ** -16
    bm = gpu_bucket(B, M, P.nnz, eps, precs)
    ids = O.bucket_ids(P.row_ptr, muf, eps, precs)["ids"]
    stored, _, _ = O.bucket_store(P.row_ptr, P.col, muf, ids, precs)
    aref, astored = _oracle_A(A, eps, precs)
    S = O.System(A, P.row_ptr, P.col, stored, ids, precs, astored, aref["ids"])
    r = O.residual_dd(A, O.spmv_prec(P.row_ptr, P.col, muf, "fp32", wl["b"]), wl["b"])
    k = 8
    d_ref, it_ref, _ = O.gmres(S, r, ug, ug, 0.0, k)
    Ah = B.matrix_create(B.DeviceCSR.from_host(A))
    ba = _bucket_A(B, Ah, A.nnz, eps, precs)
    d = torch.empty(A.n, dtype=torch.float64, device="cuda")
    info = B.gmres_b(Ah, ba["BA"], bm["BM"], dev(r), d, ug, B.opts(tau=0.0, kmax=k))
    assert info["gmres_iters"] == [k] and it_ref == k
    assert np.linalg.norm(host(d) - d_ref) <= tol * np.linalg.norm(d_ref)


@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_gmres_ir_bucketed_A_matches_oracle(B, wl):
    A, P = wl["A"], wl["pattern"]
    for eps in [2.0 ** -37, 2.0 ** -16]:
        g = gpu_build(B, wl)
        bm = gpu_bucket(B, g["M"], P.nnz, eps, wl["precs"])
        Ah = B.matrix_create(g["A"])
        BA, ainfo = B.bucket_A(Ah, eps, wl["precs"])
        x = torch.empty(A.n, dtype=torch.float64, device="cuda")
        info = B.gmres_ir_solve_hb(Ah, BA, dev(wl["b"]), bm["BM"], g["M"], x, tol=wl["tau"])
        xg = host(x)
        ref = O.solve(wl, bucket_eps=eps, bucket_A=True)
        xt = wl["x_true"]
        assert info["status"] == 0, info
        fe_g = np.abs(xg - xt).max() / np.abs(xt).max()
        fe_o = np.abs(ref["x"] - xt).max() / np.abs(xt).max()
        assert fe_g <= 1e-10 and fe_o <= 1e-10
        assert np.abs(xg - ref["x"]).max() <= 1e-12 * np.abs(ref["x"]).max()
        assert abs(info["ir_steps"] - ref["steps"]) <= 1
        # counts: the same bars as the unbucketed solve (the u_g dot-product order)
        for i, (a, c) in enumerate(zip(info["gmres_iters"], ref["its"])):
            assert abs(a - c) <= (max(2, 0.1 * c) if i == 0 else max(4, 0.2 * c)), (i, a, c)


@pytest.mark.parametrize("wl", WLS[:3], ids=IDS[:3])
def test_ir_single_fp64_bucket_equals_up_fp64(B, wl):
    """One fp64 bucket of A is A in u_p = fp64: the two IR solves take the same
    operations in the same order and give the same bits."""
    A, P = wl["A"], wl["pattern"]
    g = gpu_build(B, wl)
    bm = gpu_bucket(B, g["M"], P.nnz, 2.0 ** -16, wl["precs"])
    Ah = B.matrix_create(g["A"])
    BA, _ = B.bucket_A(Ah, 2.0 ** -16, ["fp64"])
    x1 = torch.empty(A.n, dtype=torch.float64, device="cuda")
    x2 = torch.empty_like(x1)
    i1 = B.gmres_ir_solve_hb(Ah, BA, dev(wl["b"]), bm["BM"], g["M"], x1, u_g="fp64", tol=wl["tau"])
    i2 = B.gmres_ir_solve(Ah, dev(wl["b"]), bm["BM"], g["M"], x2, u_g="fp64", u_p="fp64", tol=wl["tau"])
    assert i1["gmres_iters"] == i2["gmres_iters"]
    assert torch.equal(x1, x2)


def test_bucket_A_rejects_bad_handle(B):
    with pytest.raises(Exception):
        B.bucket_A(B.AHandle(0), 2.0 ** -16, ["fp32"])


def test_bucketed_A_of_another_size_rejected(B):
    """A bucketed matrix with a different number of rows is refused before any
    launch, and the context stays usable."""
    wl0, wl1 = WLS[0], WLS[1]
    A0 = wl0["A"]
    Ah0 = B.matrix_create(B.DeviceCSR.from_host(A0))
    Ah1 = B.matrix_create(B.DeviceCSR.from_host(wl1["A"]))
    BA1, _ = B.bucket_A(Ah1, 2.0 ** -16, ["fp64"])
    BA0, _ = B.bucket_A(Ah0, 2.0 ** -16, ["fp64"])
    g = gpu_build(B, wl0)
    bm = gpu_bucket(B, g["M"], wl0["pattern"].nnz, 2.0 ** -16, wl0["precs"])
    r = dev(wl0["b"])
    d = torch.empty(A0.n, dtype=torch.float64, device="cuda")
    with pytest.raises(Exception):
        B.gmres_b(Ah0, BA1, bm["BM"], r, d)
    x = torch.empty(A0.n, dtype=torch.float64, device="cuda")
    with pytest.raises(Exception):
        B.gmres_ir_solve_hb(Ah0, BA1, r, bm["BM"], g["M"], x, tol=wl0["tau"])
    info = B.gmres_ir_solve_hb(Ah0, BA0, r, bm["BM"], g["M"], x, tol=wl0["tau"])
    assert info["status"] == 0
