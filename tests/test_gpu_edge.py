"""GPU edge cases through the C-ABI: tiny and ragged sizes, degenerate
buckets, zero right-hand side, malformed input rejected on the host side
before any kernel indexes through it, non-finite data, forced kmax, and
run-to-run determinism."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import dev, gpu_bucket, gpu_build, host, lib, oracle_M
from paper_2307_03914_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    return lib()


def _wl(A, P=None, **kw):
    x, b = W.rhs(A)
    wl = dict(name="edge", A=A, pattern=P or W.pattern_of(A), x_true=x, b=b, spai_eps=0.3,
              precs=["fp64", "fp32", "fp16"], tau=1e-4, bucket_eps=2.0 ** -16, u_g="fp32", u_p="fp32")
    wl.update(kw)
    return wl


def _solve(B, wl, eps=2.0 ** -16, precs=None, o=None, b=None):
    g = gpu_build(B, wl)
    bk = gpu_bucket(B, g["M"], wl["pattern"].nnz, eps, precs or wl["precs"])
    x = torch.zeros(wl["A"].n, dtype=torch.float64, device="cuda")
    info = B.gmres_ir_solve(g["A"], dev(wl["b"] if b is None else b), bk["BM"], g["M"], x, tol=wl["tau"],
                            o=o)
    return host(x), info, g, bk


def test_single_unknown(B):
    A = W.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([4.0]))
    wl = _wl(A)
    x, info, g, _ = _solve(B, wl)
    assert info["status"] == 0
    assert abs(x[0] - wl["b"][0] / 4.0) <= 1e-15 * abs(x[0])
    assert g["val"][0] == np.float32(0.25)


@pytest.mark.parametrize("n", [2, 31, 32, 33, 65])
def test_ragged_1d(B, n):
    A = W.convdiff2d(n, 1, (0.5, 0.0))
    wl = _wl(A)
    x, info, g, _ = _solve(B, wl)
    ref = O.solve(wl, bucket_eps=2.0 ** -16)
    assert info["status"] == 0
    assert np.abs(x - ref["x"]).max() <= 1e-12 * np.abs(ref["x"]).max()


def test_zero_rhs(B):
    wl = _wl(W.convdiff2d(8))
    x, info, _, _ = _solve(B, wl, b=np.zeros(64))
    assert info["status"] == 0 and np.all(x == 0)


def test_diagonal_pattern(B):
    A = W.convdiff2d(10)
    P = W.CSR(A.n, np.arange(A.n + 1, dtype=np.int32), np.arange(A.n, dtype=np.int32), None)
    wl = _wl(A, P)
    x, info, g, _ = _solve(B, wl)
    ref = O.spai(A, P, 0.3)
    assert np.allclose(g["val"], ref["mval"], rtol=1e-6)
    assert info["status"] == 0
    assert np.abs(x - wl["x_true"]).max() <= 1e-10


def test_empty_and_fully_dropped_buckets(B):
    wl = _wl(W.convdiff3d(6), precs=["fp64", "fp32", "fp16", "e4m3"])
    M, muf = oracle_M(B, wl)
    P = wl["pattern"]
    # eps so small that every entry lands in the fp64 bucket: three empty buckets
    bk = gpu_bucket(B, M, P.nnz, 2.0 ** -53, wl["precs"])
    assert bk["info"]["nnz_k"][1:] == [0, 0, 0]
    xin = np.random.default_rng(0).uniform(-1, 1, P.n)
    y = torch.empty(P.n, dtype=torch.float64, device="cuda")
    B.apply(bk["BM"], dev(xin), y)
    ids = O.bucket_ids(P.row_ptr, muf, 2.0 ** -53, wl["precs"])["ids"]
    stored, _, _ = O.bucket_store(P.row_ptr, P.col, muf, ids, wl["precs"])
    ref = O.bspmv(P.row_ptr, P.col, stored, ids, wl["precs"], xin)
    assert np.array_equal(host(y), ref)
    # eps = 1 with (fp64, drop): everything is dropped and M v = 0
    bk = gpu_bucket(B, M, P.nnz, 1.0, ["fp64", "drop"])
    assert bk["info"]["nnz_k"] == [0, P.nnz] and bk["info"]["storage_pct"] == 0.0
    B.apply(bk["BM"], dev(xin), y)
    assert np.all(host(y) == 0)


def test_malformed_input_is_rejected(B):
    A = W.convdiff2d(6)
    bad = W.CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val.copy())
    bad.col[5] = A.n + 7  # out of range
    with pytest.raises(B.BspaiError) as e:
        B.matrix_create(B.DeviceCSR.from_host(bad))
    assert e.value.status == B.ERR_INVALID
    unsorted = W.CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val.copy())
    unsorted.col[[0, 1]] = unsorted.col[[1, 0]]
    with pytest.raises(B.BspaiError):
        B.bspai_build(B.DeviceCSR.from_host(unsorted), B.DeviceCSR.from_host(W.pattern_of(A), with_values=False),
                      0.3)
    g = gpu_build(B, _wl(A))
    with pytest.raises(B.BspaiError) as e:
        B.bspai_bucket(g["M"], 2.0 ** -20, ["fp32", "fp64"])
    assert e.value.status == B.ERR_INVALID
    with pytest.raises(B.BspaiError):
        B.bspai_bucket(g["M"], 2.0 ** -20, ["fp64", "e4m3", "e4m3"])
    # the context is still usable
    x, info, _, _ = _solve(B, _wl(A))
    assert info["status"] == 0


def test_nonfinite_rhs_reported(B):
    wl = _wl(W.convdiff2d(6))
    b = wl["b"].copy()
    b[3] = np.nan
    _, info, _, _ = _solve(B, wl, b=b)
    assert info["status"] == B.NONFINITE


def test_forced_kmax_and_imax(B):
    wl = _wl(W.convdiff2d(16))
    _, info, _, _ = _solve(B, wl, o=B.opts(tau=1e-4, kmax=1, i_max=3))
    assert info["status"] == B.NOT_CONVERGED
    assert info["gmres_iters"] == [1, 1, 1] and info["ir_steps"] == 3


def test_deterministic(B):
    wl = W.workload("convdiff3d", grid=10)
    x1, i1, _, _ = _solve(B, wl)
    x2, i2, _, _ = _solve(B, wl)
    assert np.array_equal(x1, x2) and i1["gmres_iters"] == i2["gmres_iters"]


def test_fp64_comparator_path(B):
    """q = 1 {fp64}, u_g = u_p = fp64: plain SPAI-GMRES-IR with the paper's u_g = u_p = u."""
    wl = W.workload("convdiff2d")
    M, muf = oracle_M(B, wl)
    bk = gpu_bucket(B, M, wl["pattern"].nnz, 2.0 ** -53, ["fp64"])
    x = torch.empty(wl["A"].n, dtype=torch.float64, device="cuda")
    info = B.gmres_ir_solve(B.DeviceCSR.from_host(wl["A"]), dev(wl["b"]), bk["BM"], M, x, u_g="fp64", u_p="fp64",
                            tol=1e-8)
    xg = host(x)
    assert info["status"] == 0
    assert np.abs(xg - wl["x_true"]).max() <= 1e-12
    S = O.System(wl["A"], wl["pattern"].row_ptr, wl["pattern"].col, muf, np.zeros(wl["pattern"].nnz, np.int8),
                 ["fp64"])
    ref = O.gmres_ir(S, muf, wl["b"], "fp64", "fp64", 1e-8, 500, 10)
    assert np.abs(xg - ref["x"]).max() <= 1e-12 * np.abs(ref["x"]).max()
    assert info["gmres_iters"][0] == ref["its"][0]


def test_barrier_wait_runs_out_and_context_survives(B):
    """Failure detection without a fault: a grid barrier that nothing releases
    gives up after its time limit, the call reports BSPAI_TIMEOUT, and the next
    barrier and a full solve on the same context still work."""
    st, ms = B.barrier_selftest(8, hold=False, timeout_s=1.0)
    assert st == B.OK and ms < 500.0
    st, ms = B.barrier_selftest(8, hold=True, timeout_s=0.25)
    assert st == B.TIMEOUT
    assert 200.0 <= ms <= 5000.0, ms
    assert "timed out" in B.last_error()
    st, _ = B.barrier_selftest(152, hold=False, timeout_s=1.0)
    assert st == B.OK
    wl = _wl(W.convdiff2d(16))
    x, info, _, _ = _solve(B, wl)
    assert info["status"] == B.OK
    xt = wl["x_true"]
    assert np.abs(x - xt).max() / np.abs(xt).max() <= 1e-10
