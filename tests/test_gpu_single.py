"""GPU parity of the (u_f, u, u_r) = (single, single, double) setting (Section
4, Table 4): working precision u = fp32 (x, r and the correction held in
fp32), the residual in plain fp64, buckets {single, half, drop} with
bucket_eps in {2^-24, 2^-18}, u_g = u_p = single, tau = 1e-4.

Bars:
  * r = b - A x in u_r in {Dot2, fp64}, stored in u in {fp64, fp32}: bit-exact;
  * refinement: x is fp32-valued; both sides reach forward error <= 2u
    (u = 2^-24, the limiting accuracy when u_r = u^2), so they agree within 4u
    in the infinity norm; the same number of refinement steps within one and
    first-step GMRES counts within max(2, 10 %) (the u_g dot-product order
    differs, as in the u = fp64 tests).
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import dev, gpu_bucket, gpu_build, host, lib, small_workloads

pytestmark = pytest.mark.gpu

WLS = small_workloads()
IDS = [f"{w['name']}-{w['A'].n}" for w in WLS]
U = 2.0 ** -24
PRECS = ["fp32", "fp16", "drop"]


@pytest.fixture(scope="module")
def B():
    return lib()


@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_residual_prec_bitexact(B, wl):
    A = wl["A"]
    rng = np.random.default_rng(31)
    x = (wl["x_true"] + rng.normal(0, 1e-6, A.n)).astype(np.float32).astype(np.float64)
    Ah = B.matrix_create(B.DeviceCSR.from_host(A))
    r = torch.empty(A.n, dtype=torch.float64, device="cuda")
    for u_r, fn in [("dd", O.residual_dd), ("fp64", O.residual_fp64)]:
        for u in ["fp64", "fp32"]:
            B.residual_prec(Ah, dev(x), dev(wl["b"]), r, u_r=u_r, u=u)
            ref = fn(A, x, wl["b"])
            if u == "fp32":
                ref = O.round_to(ref, "fp32")
            assert np.array_equal(host(r), ref), (u_r, u)


def _check_against_oracle(info, xg, ref, wl):
    xt = wl["x_true"]
    assert info["status"] == 0, info
    assert np.array_equal(xg, xg.astype(np.float32).astype(np.float64))
    fe_g = np.abs(xg - xt).max() / np.abs(xt).max()
    fe_o = np.abs(ref["x"] - xt).max() / np.abs(xt).max()
    assert fe_g <= 2 * U and fe_o <= 2 * U, (fe_g, fe_o)
    assert np.abs(xg - ref["x"]).max() <= 4 * U * np.abs(ref["x"]).max()
    assert abs(info["ir_steps"] - ref["steps"]) <= 1
    assert abs(info["gmres_iters"][0] - ref["its"][0]) <= max(2, 0.1 * ref["its"][0])


@pytest.mark.parametrize("eps", [2.0 ** -24, 2.0 ** -18])
@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_ir_single_single_double_matches_oracle(B, wl, eps):
    A, P = wl["A"], wl["pattern"]
    g = gpu_build(B, wl)
    bm = gpu_bucket(B, g["M"], P.nnz, eps, PRECS)
    x = torch.empty(A.n, dtype=torch.float64, device="cuda")
    info = B.gmres_ir_solve(g["A"], dev(wl["b"]), bm["BM"], g["M"], x, u="fp32", u_r="fp64", u_g="fp32",
                            u_p="fp32", tol=1e-4)
    ref = O.solve(wl, bucket_eps=eps, precs=PRECS, u="fp32", u_r="fp64", ug="fp32", up="fp32", tau=1e-4)
    _check_against_oracle(info, host(x), ref, wl)


@pytest.mark.parametrize("wl", WLS[:3], ids=IDS[:3])
def test_ir_single_with_bucketed_A_matches_oracle(B, wl):
    """u = fp32 together with A v through A's own buckets (eq. nbe2)."""
    A, P = wl["A"], wl["pattern"]
    eps = 2.0 ** -18
    g = gpu_build(B, wl)
    bm = gpu_bucket(B, g["M"], P.nnz, eps, PRECS)
    Ah = B.matrix_create(g["A"])
    BA, _ = B.bucket_A(Ah, eps, PRECS)
    x = torch.empty(A.n, dtype=torch.float64, device="cuda")
    info = B.gmres_ir_solve_hb(Ah, BA, dev(wl["b"]), bm["BM"], g["M"], x, u="fp32", u_r="fp64", u_g="fp32",
                               tol=1e-4)
    ref = O.solve(wl, bucket_eps=eps, precs=PRECS, u="fp32", u_r="fp64", ug="fp32", up="fp32", tau=1e-4,
                  bucket_A=True)
    _check_against_oracle(info, host(x), ref, wl)


def test_given_x0_is_held_in_fp32(B):
    wl = WLS[0]
    A, P = wl["A"], wl["pattern"]
    g = gpu_build(B, wl)
    bm = gpu_bucket(B, g["M"], P.nnz, 2.0 ** -24, PRECS)
    x0 = wl["x_true"] + np.random.default_rng(3).normal(0, 1e-3, A.n)
    x = dev(x0)
    info = B.gmres_ir_solve(g["A"], dev(wl["b"]), bm["BM"], None, x, u="fp32", u_r="fp64", u_g="fp32",
                            u_p="fp32", tol=1e-4, o=B.opts(tau=1e-4, x0_given=True))
    xg = host(x)
    assert info["status"] == 0
    assert np.array_equal(xg, xg.astype(np.float32).astype(np.float64))
    assert np.abs(xg - wl["x_true"]).max() / np.abs(wl["x_true"]).max() <= 2 * U


def test_unsupported_working_precision_rejected(B):
    wl = WLS[0]
    A, P = wl["A"], wl["pattern"]
    g = gpu_build(B, wl)
    bm = gpu_bucket(B, g["M"], P.nnz, 2.0 ** -24, PRECS)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(Exception):
        B.gmres_ir_solve(g["A"], dev(wl["b"]), bm["BM"], g["M"], x, u="fp16", u_r="fp64", tol=1e-4)
    Ah = B.matrix_create(g["A"])
    with pytest.raises(Exception):
        B.residual_prec(Ah, x, dev(wl["b"]), x, u_r="fp32", u="fp64")
