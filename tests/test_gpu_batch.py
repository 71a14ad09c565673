"""Batched BSPAI-GMRES-IR (many independent systems and right-hand sides per
launch): per-system bucketing bit-exact against the oracle bucketing each
system alone, every (system, right-hand side) solution within 1e-12 of the
oracle's own solve of that system, and the full 512-system x 32-RHS batch to
forward error <= 1e-10 for every pair."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import dev, host, lib
from paper_2307_03914_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    return lib()


def _system_wl(bw, s):
    A = bw["mats"][s]
    return dict(A=A, pattern=W.pattern_of(A), spai_eps=bw["spai_eps"], precs=bw["precs"], u_g="fp32", u_p="fp32",
                tau=bw["tau"], b=None, x_true=None)


def _gpu_batch(B, bw, eps=None):
    A = B.DeviceCSR.from_host(bw["A"])
    P = B.DeviceCSR.from_host(bw["pattern"], with_values=False)
    Ah = B.matrix_create(A)
    M, binfo = B.bspai_build(A, P, bw["spai_eps"])
    row_off = dev(bw["row_off"])
    BM, kinfo = B.bspai_bucket_batched(M, row_off, bw["bucket_eps"] if eps is None else eps, bw["precs"])
    Bd = dev(bw["B"].reshape(-1))
    X = torch.zeros_like(Bd)
    npairs = len(bw["mats"]) * bw["nrhs"]
    st = torch.empty(npairs, dtype=torch.int32, device="cuda")
    it = torch.empty(npairs, dtype=torch.int32, device="cuda")
    info = B.gmres_ir_solve_batched(Ah, row_off, bw["nrhs"], Bd, BM, M, X, tol=bw["tau"], pair_status=st,
                                    pair_iters=it)
    return dict(X=X, info=info, status=host(st), iters=host(it), M=M, BM=BM, kinfo=kinfo, row_off=row_off)


def test_batched_bucketing_matches_per_system_oracle(B):
    bw = W.batch_workload(nsys=7, nrhs=2, nmin=60, nmax=1500, seed=3)
    # the oracle's M of every system, stacked and handed to the library
    mufs = []
    for s in range(len(bw["mats"])):
        wl = _system_wl(bw, s)
        mufs.append(O.round_to(O.spai(wl["A"], wl["pattern"], wl["spai_eps"])["mval"], "fp32"))
    P = bw["pattern"]
    Mcsr = B.DeviceCSR(P.n, dev(P.row_ptr), dev(P.col), dev(np.concatenate(mufs)))
    M = B.M_create(Mcsr)
    row_off = dev(bw["row_off"])
    for precs, eps in [(bw["precs"], 2.0 ** -16), (["fp64", "fp32", "fp16", "e4m3", "drop"], 2.0 ** -12)]:
        BM, _ = B.bspai_bucket_batched(M, row_off, eps, precs)
        ids, stored = B.bucket_export(BM, P.nnz)
        ids, stored = host(ids), host(stored)
        off = 0
        for s, m in enumerate(bw["mats"]):
            nnz = m.nnz
            ref = O.bucket_ids(m.row_ptr, mufs[s], eps, precs)
            st, _, _ = O.bucket_store(m.row_ptr, m.col, mufs[s], ref["ids"], precs)
            assert np.array_equal(ids[off:off + nnz], ref["ids"]), (s, precs)
            assert np.array_equal(stored[off:off + nnz], st), (s, precs)
            off += nnz
        # the product on the stacked vector equals each system's own product
        x = np.random.default_rng(1).uniform(-1, 1, P.n)
        y = torch.empty(P.n, dtype=torch.float64, device="cuda")
        B.apply(BM, dev(x), y)
        yh = host(y)
        ro = bw["row_off"]
        for s, m in enumerate(bw["mats"]):
            ref = O.bucket_ids(m.row_ptr, mufs[s], eps, precs)
            st, _, _ = O.bucket_store(m.row_ptr, m.col, mufs[s], ref["ids"], precs)
            yr = O.bspmv(m.row_ptr, m.col, st, ref["ids"], precs, x[ro[s]:ro[s] + m.n])
            assert np.array_equal(yh[ro[s]:ro[s] + m.n], yr), s


def test_batched_solve_matches_oracle_per_pair(B):
    bw = W.batch_workload(nsys=6, nrhs=3, nmin=60, nmax=1200, seed=5)
    g = _gpu_batch(B, bw)
    assert g["info"]["status"] == 0 and g["info"]["converged"] == g["info"]["pairs"]
    assert np.all(g["status"] > 0)
    n = bw["A"].n
    X = host(g["X"]).reshape(bw["nrhs"], n)
    ro = bw["row_off"]
    for s, m in enumerate(bw["mats"]):
        wl = _system_wl(bw, s)
        for r in range(bw["nrhs"]):
            wl["b"] = bw["B"][r, ro[s]:ro[s] + m.n]
            xt = bw["X_true"][r, ro[s]:ro[s] + m.n]
            ref = O.solve(wl, bucket_eps=bw["bucket_eps"])
            xg = X[r, ro[s]:ro[s] + m.n]
            assert np.abs(xg - ref["x"]).max() <= 1e-12 * np.abs(ref["x"]).max(), (s, r)
            assert np.abs(xg - xt).max() / np.abs(xt).max() <= 1e-10
            # GMRES steps summed over the refinement steps within a few steps (the late
            # steps' counts move with the u_g summation order, see test_gpu_parity)
            assert abs(g["iters"][r * len(bw["mats"]) + s] - sum(ref["its"])) <= max(4, 0.15 * sum(ref["its"]))
        # padding rows stay zero
        assert np.all(X[:, ro[s] + m.n:ro[s + 1]] == 0)


def test_batch_of_one_equals_single_solve(B):
    bw = W.batch_workload(nsys=1, nrhs=1, nmin=900, nmax=1000, seed=7)
    g = _gpu_batch(B, bw)
    m = bw["mats"][0]
    A = B.DeviceCSR.from_host(m)
    P = B.DeviceCSR.from_host(W.pattern_of(m), with_values=False)
    M, _ = B.bspai_build(A, P, bw["spai_eps"])
    BM, _ = B.bspai_bucket(M, bw["bucket_eps"], bw["precs"])
    x = torch.empty(m.n, dtype=torch.float64, device="cuda")
    B.gmres_ir_solve(A, dev(bw["B"][0, :m.n]), BM, M, x, tol=bw["tau"])
    xb = host(g["X"])[:m.n]
    assert np.abs(xb - host(x)).max() <= 1e-12 * np.abs(host(x)).max()


def test_batch_rejects_unaligned_offsets(B):
    bw = W.batch_workload(nsys=2, nrhs=1, nmin=100, nmax=200, seed=9)
    A = B.DeviceCSR.from_host(bw["A"])
    P = B.DeviceCSR.from_host(bw["pattern"], with_values=False)
    M, _ = B.bspai_build(A, P, 0.3)
    bad = bw["row_off"].copy()
    bad[1] -= 1
    with pytest.raises(B.BspaiError) as e:
        B.bspai_bucket_batched(M, dev(bad), 2.0 ** -16, bw["precs"])
    assert e.value.status == B.ERR_INVALID


def test_full_batch_512_systems_32_rhs(B):
    bw = W.batch_workload()
    g = _gpu_batch(B, bw)
    info = g["info"]
    assert info["pairs"] == 512 * 32 and info["converged"] == info["pairs"], info
    n = bw["A"].n
    X = g["X"].reshape(bw["nrhs"], n)
    Xt = dev(bw["X_true"])
    err = (X - Xt).abs()
    ro = bw["row_off"]
    worst = 0.0
    for s, m in enumerate(bw["mats"]):
        e = err[:, ro[s]:ro[s] + m.n].amax(dim=1)
        t = Xt[:, ro[s]:ro[s] + m.n].abs().amax(dim=1)
        worst = max(worst, float((e / t).max()))
    assert worst <= 1e-10, worst
    print("batch:", info, f"worst forward error {worst:.2e}")
