"""Element-wise parity of every modified Gram-Schmidt kernel instance the GMRES
solves can pick (Alg 3.1, GMRES line; Section 3 analyses MGS-GMRES) against the
oracle's GMRES, at the problem sizes where each instance runs.

The instance depends on the order n (rows of the new Krylov vector each block
holds on chip): a sweep of 3D convection-diffusion grids reaches every one of
them, and each case asserts through bspai_gmres_plan which one ran.  The
largest case is the benchmark's own 128^3 workload with its bucketing
(eps = 2^-10, buckets {fp64, fp32, fp16, e4m3}), where k_mgs_res2 with 16 row
pairs per thread of a 512-thread block runs on 128 blocks, its reductions
polled by bulk copies.

Both sides get the oracle's M (fp64 SPAI rounded to u_f = fp32), bucketed by
each side (bit-exact, checked elsewhere), and the same residual r of
x0 = M b; GMRES runs a fixed number of steps (tau = 0).  Bar: the corrections
agree element-wise within 1e-4 (u_g = fp32) / 1e-10 (u_g = fp64) of their
largest entry -- the two sides add the u_g dot products in different orders
(a fixed tree on the GPU, pairwise in the oracle), which the paper leaves
open -- and the GMRES residual estimates |g_k| / beta agree to the same
relative level."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import dev, gpu_bucket, host, lib
from paper_2307_03914_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BENCH_EPS = 2.0 ** -10
TOL = {"fp32": 1e-4, "fp64": 1e-10}

# (grid, u_g, kernel, rows or row pairs per thread, block threads, how warp 0 reads the
# reduction slots: by loads, or by bulk copies from 16 KB of a vector per block); 152 SMs
SWEEP = [
    (40, "fp32", "k_mgs_res", 1, 1024, "loads"),     # n = 64,000: a chunk of <= 1024 rows per block
    (48, "fp32", "k_mgs_res2", 1, 1024, "loads"),    # n = 110,592
    (64, "fp32", "k_mgs_res2", 2, 1024, "bulk"),     # n = 262,144
    (80, "fp32", "k_mgs_res2", 4, 1024, "bulk"),     # n = 512,000
    (88, "fp32", "k_mgs_res2", 12, 512, "bulk"),     # n = 681,472
    (94, "fp32", "k_mgs_res2", 14, 512, "bulk"),     # n = 830,584
    (100, "fp32", "k_mgs_res2", 16, 512, "bulk"),    # n = 1,000,000
    (40, "fp64", "k_mgs_res", 1, 1024, "loads"),
    (48, "fp64", "k_mgs_res", 2, 1024, "loads"),     # 13.8 KB of a vector per block
    (64, "fp64", "k_mgs_res", 4, 1024, "bulk"),
    (80, "fp64", "k_mgs_res", 8, 1024, "bulk"),
    (110, "fp64", "k_mgs", 0, 512, "loads"),         # n = 1,331,000: beyond on-chip rows, the streaming kernel
]


@pytest.fixture(scope="module")
def B():
    b = lib()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    if sms != 152:
        pytest.skip(f"instance table written for 152 SMs (this device has {sms})")
    return b


def _case(B, grid, eps, precs):
    wl = W.workload("convdiff3d", grid=grid)
    A, P = wl["A"], wl["pattern"]
    sp = O.spai(A, P, wl["spai_eps"])
    muf = O.round_to(sp["mval"], "fp32")
    Mh = B.M_create(B.DeviceCSR(P.n, dev(P.row_ptr.astype(np.int32)), dev(P.col.astype(np.int32)), dev(muf)))
    bk = gpu_bucket(B, Mh, P.nnz, eps, precs)
    ids = O.bucket_ids(P.row_ptr, muf, eps, precs)["ids"]
    stored, _, _ = O.bucket_store(P.row_ptr, P.col, muf, ids, precs)
    S = O.System(A, P.row_ptr, P.col, stored, ids, precs)
    r = O.residual_dd(A, O.spmv_prec(P.row_ptr, P.col, muf, "fp32", wl["b"]), wl["b"])
    return wl, bk, S, r


def _compare(B, wl, bk, S, r, ug, k):
    A = wl["A"]
    d_ref, it_ref, res_ref = O.gmres(S, r, ug, ug, 0.0, k)
    Ah = B.matrix_create(B.DeviceCSR.from_host(A))
    d = torch.empty(A.n, dtype=torch.float64, device="cuda")
    info = B.gmres(Ah, bk["BM"], dev(r), d, ug, ug, B.opts(tau=0.0, kmax=k))
    assert info["gmres_iters"] == [k] and it_ref == k
    dg = host(d)
    err = np.abs(dg - d_ref).max() / np.abs(d_ref).max()
    assert err <= TOL[ug], err
    # |g_k| / ||M r||_2 (res_ref is the oracle's relative estimate)
    assert abs(info["relres"][0] - res_ref) <= 10 * TOL[ug] * res_ref, (info["relres"], res_ref)
    return err


@pytest.mark.parametrize("grid,ug,kernel,per_thread,bd,poll", SWEEP,
                         ids=[f"{g}^3-{u}-{k}<{p},{b}>-{q}" for g, u, k, p, b, q in SWEEP])
def test_mgs_instance_matches_oracle(B, grid, ug, kernel, per_thread, bd, poll):
    n = grid ** 3
    plan = B.gmres_plan(n, ug)
    assert (plan["kernel"], plan["per_thread"], plan["block_threads"], plan["poll"]) == \
        (kernel, per_thread, bd, poll), plan
    wl, bk, S, r = _case(B, grid, 2.0 ** -16, ["fp64", "fp32", "fp16", "e4m3"])
    err = _compare(B, wl, bk, S, r, ug, 16)
    print(f"{grid}^3 {ug} {kernel}<{per_thread},{bd}> x {plan['blocks']} ({poll}): max rel diff {err:.2e}")


def test_mgs_bench_instance_128(B):
    """The benchmark's configuration: 128^3, eps = 2^-10, u_g = fp32 --
    k_mgs_res2 with 16 row pairs per thread, 512 threads, 128 blocks --
    24 Arnoldi steps against the oracle."""
    plan = B.gmres_plan(128 ** 3, "fp32")
    assert plan == dict(kernel="k_mgs_res2", per_thread=16, block_threads=512, blocks=128, poll="bulk"), plan
    wl, bk, S, r = _case(B, 128, BENCH_EPS, ["fp64", "fp32", "fp16", "e4m3"])
    assert bk["info"]["nnz_k"][2] > 0 and bk["info"]["nnz_k"][3] > 0  # the fp16 + e4m3 form of M w
    err = _compare(B, wl, bk, S, r, "fp32", 24)
    print(f"128^3 fp32 k_mgs_res2<16,512> x 128: max rel diff {err:.2e}")
