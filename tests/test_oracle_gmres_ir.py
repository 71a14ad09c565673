"""Pins for the oracle's left-preconditioned MGS-GMRES and the refinement
driver (Alg 3.1), against dense linear algebra and exact arithmetic."""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2307_03914_gb300 import workloads as W


def _csr(Ad):
    S = sp.csr_matrix(Ad)
    S.sort_indices()
    return W.CSR(Ad.shape[0], S.indptr.astype(np.int32), S.indices.astype(np.int32),
                 S.data.astype(float))


def _system(orc, A, Mdense, fmts=("fp64",)):
    Mc = _csr(Mdense)
    ids = np.zeros(Mc.nnz, np.int8)
    return orc.System(A, Mc.row_ptr, Mc.col, Mc.val, ids, list(fmts))


def test_exact_inverse_preconditioner_converges_in_one_iteration(orc):
    A = W.convdiff2d(6)
    Ainv = np.linalg.inv(A.to_scipy().toarray())
    S = _system(orc, A, Ainv)
    r = np.random.default_rng(1).uniform(-1, 1, A.n)
    d, its, rel = orc.gmres(S, r, ug="fp64", up="fp64", tau=1e-10, kmax=A.n)
    assert its == 1
    assert np.allclose(d, Ainv @ r, rtol=1e-12, atol=1e-14)


def test_identity_preconditioner_full_krylov_equals_dense_solve(orc):
    A = W.random_sparse(40, 5, sigma=1.0, delta=0.3, seed=4)
    Ad = A.to_scipy().toarray()
    S = _system(orc, A, np.eye(A.n))
    r = np.random.default_rng(2).uniform(-1, 1, A.n)
    d, its, rel = orc.gmres(S, r, ug="fp64", up="fp64", tau=0.0, kmax=A.n)
    ref = np.linalg.solve(Ad, r)
    assert np.linalg.norm(d - ref) <= 1e-10 * np.linalg.cond(Ad) * np.linalg.norm(ref)


@pytest.mark.parametrize("k", [1, 3, 7])
def test_gmres_iterate_minimises_residual_over_krylov_space(orc, k):
    """GMRES(k) returns argmin ||s - MA d|| over K_k(MA, s) (Saad, Prop. 6.x);
    checked against a least-squares solve on an explicit Krylov basis."""
    A = W.convdiff2d(5)
    Ad = A.to_scipy().toarray()
    rng = np.random.default_rng(k)
    M = np.diag(1.0 / np.diag(Ad)) + 0.01 * rng.normal(size=Ad.shape) * (np.abs(Ad) > 0)
    S = _system(orc, A, M)
    r = rng.uniform(-1, 1, A.n)
    d, its, _ = orc.gmres(S, r, ug="fp64", up="fp64", tau=0.0, kmax=k)
    assert its == k
    T = M @ Ad
    s = M @ r
    K = np.empty((A.n, k))
    v = s / np.linalg.norm(s)
    for j in range(k):
        K[:, j] = v
        v = T @ v
        v /= np.linalg.norm(v)
    Q, _ = np.linalg.qr(K)
    c, *_ = np.linalg.lstsq(T @ Q, s, rcond=None)
    ref = Q @ c
    assert np.linalg.norm(d - ref) <= 1e-8 * np.linalg.norm(ref)
    # and the reported residual estimate equals the true preconditioned residual
    d2, _, rel = orc.gmres(S, r, ug="fp64", up="fp64", tau=0.0, kmax=k)
    assert abs(rel - np.linalg.norm(s - T @ d2) / np.linalg.norm(s)) <= 1e-10


def test_fp32_gmres_tracks_fp64(orc):
    """u_g = u_p = fp32 vs fp64: the corrections agree to about kappa * u_g."""
    wl = W.workload("convdiff2d", grid=10)
    A = wl["A"]
    sp_ = orc.spai(A, wl["pattern"], 0.3)
    muf = orc.round_to(sp_["mval"], "fp32")
    bk = orc.bucket_ids(wl["pattern"].row_ptr, muf, 2.0 ** -53, ["fp64"])
    S = orc.System(A, wl["pattern"].row_ptr, wl["pattern"].col, muf, bk["ids"], ["fp64"])
    r = wl["b"]
    d64, it64, _ = orc.gmres(S, r, "fp64", "fp64", 1e-6, 200)
    d32, it32, _ = orc.gmres(S, r, "fp32", "fp32", 1e-6, 200)
    kap = np.linalg.cond(A.to_scipy().toarray(), np.inf)
    assert np.abs(d32 - d64).max() <= 50 * kap * 2.0 ** -24 * np.abs(d64).max()
    assert abs(it32 - it64) <= 3


def _exact_solve(Ad, b):
    n = len(b)
    M = [[Fraction(Ad[i, j]) for j in range(n)] + [Fraction(b[i])] for i in range(n)]
    for c in range(n):
        piv = max(range(c, n), key=lambda i: abs(M[i][c]))
        M[c], M[piv] = M[piv], M[c]
        for i in range(c + 1, n):
            f = M[i][c] / M[c][c]
            for j in range(c, n + 1):
                M[i][j] -= f * M[c][j]
    x = [Fraction(0)] * n
    for i in range(n - 1, -1, -1):
        x[i] = (M[i][n] - sum(M[i][j] * x[j] for j in range(i + 1, n))) / M[i][i]
    return x


def test_ir_reaches_working_precision_on_tiny_system(orc):
    """kappa_inf(A) well below u^(-1/3) u_f^(-2/3): forward error reaches the
    level of u against the exact rational solution (Section 1, Alg 3.1)."""
    wl = W.workload("convdiff2d", grid=4)
    A = wl["A"]
    Ad = A.to_scipy().toarray()
    kap = np.linalg.cond(Ad, np.inf)
    assert kap <= (2.0 ** -53) ** (-1 / 3) * (2.0 ** -24) ** (-2 / 3)
    out = orc.solve(wl)
    xe = _exact_solve(Ad, wl["b"])
    xr = np.array([float(v) for v in xe])
    fe = np.abs(out["x"] - xr).max() / np.abs(xr).max()
    condx = np.abs(np.linalg.inv(Ad)) @ np.abs(Ad) @ np.abs(xr)
    assert fe <= 4 * condx.max() / np.abs(xr).max() * 2.0 ** -53
    assert out["nbe"][-1] <= 2.0 ** -53 or out["stop"] in (2, 3)


@pytest.mark.parametrize("name,grid", [("convdiff2d", 32), ("convdiff3d", 8)])
def test_ir_solves_workloads_to_forward_error_1e10(orc, name, grid):
    wl = W.workload(name, grid=grid)
    out = orc.solve(wl)
    xt = wl["x_true"]
    fe = np.abs(out["x"] - xt).max() / np.abs(xt).max()
    assert fe <= 1e-10
    assert out["steps"] >= 2
    # bucketing with q = 1 is plain SPAI-GMRES-IR: same iterates as the unbucketed M
    out1 = orc.solve(wl, precs=["fp64"])
    assert np.abs(out1["x"] - xt).max() / np.abs(xt).max() <= 1e-10


def _a_buckets(orc, A, eps, fmts):
    ids = orc.bucket_ids(A.row_ptr, A.val, eps, fmts)["ids"]
    stored, _, _ = orc.bucket_store(A.row_ptr, A.col, A.val, ids, fmts)
    return stored, ids


def test_single_fp64_bucket_of_A_is_A_in_fp64(orc):
    """A v through one fp64 bucket of A (eq. nbe2 with q = 1) is A v with u_p =
    fp64: the GMRES iterates agree to the last bit."""
    A = W.convdiff2d(7)
    Ad = A.to_scipy().toarray()
    M = np.diag(1.0 / np.diag(Ad))
    Mc = _csr(M)
    mids = np.zeros(Mc.nnz, np.int8)
    a_stored, a_ids = _a_buckets(orc, A, 2.0 ** -20, ["fp64"])
    assert np.array_equal(a_stored, A.val) and not a_ids.any()
    r = np.random.default_rng(7).uniform(-1, 1, A.n)
    S0 = orc.System(A, Mc.row_ptr, Mc.col, Mc.val, mids, ["fp64"])
    S1 = orc.System(A, Mc.row_ptr, Mc.col, Mc.val, mids, ["fp64"], a_stored, a_ids)
    d0, i0, _ = orc.gmres(S0, r, ug="fp64", up="fp64", tau=0.0, kmax=9)
    d1, i1, _ = orc.gmres(S1, r, ug="fp64", up="fp64", tau=0.0, kmax=9)
    assert i0 == i1 == 9 and np.array_equal(d0, d1)


@pytest.mark.parametrize("k", [2, 5])
def test_gmres_with_bucketed_A_minimises_over_perturbed_krylov_space(orc, k):
    """With A bucketed into {fp64, drop}, A v inside GMRES is A~ v where A~
    keeps the fp64 bucket and zeroes the dropped entries; GMRES(k) then
    returns argmin ||s - M A~ d|| over K_k(M A~, s), s = M r."""
    A = W.random_sparse(60, 6, sigma=2.0, delta=0.3, seed=11)
    fmts = ["fp64", "drop"]
    a_stored, a_ids = _a_buckets(orc, A, 2.0 ** -14, fmts)
    assert (a_ids == 1).any() and (a_ids == 0).any()
    At = sp.csr_matrix((np.where(a_ids == 0, a_stored, 0.0), A.col, A.row_ptr), shape=(A.n, A.n)).toarray()
    Ad = A.to_scipy().toarray()
    assert not np.array_equal(At, Ad)
    M = np.diag(1.0 / np.diag(Ad))
    Mc = _csr(M)
    S = orc.System(A, Mc.row_ptr, Mc.col, Mc.val, np.zeros(Mc.nnz, np.int8), fmts, a_stored, a_ids)
    r = np.random.default_rng(k).uniform(-1, 1, A.n)
    d, its, _ = orc.gmres(S, r, ug="fp64", up="fp64", tau=0.0, kmax=k)
    assert its == k
    T = M @ At
    s = M @ r
    K = np.empty((A.n, k))
    v = s.copy()
    for j in range(k):
        K[:, j] = v / np.linalg.norm(v)
        v = T @ K[:, j]
    c, *_ = np.linalg.lstsq(T @ K, s, rcond=None)
    ref = K @ c
    assert np.linalg.norm(d - ref) <= 1e-12 * np.linalg.norm(ref)
    # and not the minimiser over the unperturbed operator
    T0 = M @ Ad
    K0 = np.empty((A.n, k))
    v = s.copy()
    for j in range(k):
        K0[:, j] = v / np.linalg.norm(v)
        v = T0 @ K0[:, j]
    c0, *_ = np.linalg.lstsq(T0 @ K0, s, rcond=None)
    assert np.linalg.norm(d - K0 @ c0) > 1e-4 * np.linalg.norm(ref)


@pytest.mark.parametrize("name,grid", [("convdiff2d", 32), ("convdiff3d", 8)])
def test_ir_with_bucketed_A_reaches_forward_error_1e10(orc, name, grid):
    """Refinement with A v in the bucketed precisions still converges: the
    residual uses A itself, so the perturbation of A inside GMRES only slows
    the correction solves down (Section 3, fe2)."""
    wl = W.workload(name, grid=grid)
    for eps in [2.0 ** -16, 2.0 ** -10]:
        out = orc.solve(wl, bucket_eps=eps, bucket_A=True)
        xt = wl["x_true"]
        assert np.abs(out["x"] - xt).max() / np.abs(xt).max() <= 1e-10


SSD = dict(precs=["fp32", "fp16", "drop"], u="fp32", u_r="fp64", ug="fp32", up="fp32", tau=1e-4)


@pytest.mark.parametrize("name,grid", [("convdiff2d", 32), ("convdiff3d", 8)])
@pytest.mark.parametrize("eps", [2.0 ** -24, 2.0 ** -18])
def test_ir_single_single_double_reaches_single_accuracy(orc, name, grid, eps):
    """(u_f, u, u_r) = (single, single, double) with buckets {single, half, drop}
    (Section 4, Table 4 setting): x is held in fp32 and the forward error
    reaches the level of u = 2^-24 (u_r = u^2 makes cond(A, x) u_r negligible
    for these systems, so the limiting accuracy is u itself)."""
    wl = W.workload(name, grid=grid)
    out = orc.solve(wl, bucket_eps=eps, **SSD)
    x, xt = out["x"], wl["x_true"]
    assert np.array_equal(x, x.astype(np.float32).astype(np.float64))
    assert np.abs(x - xt).max() / np.abs(xt).max() <= 2 * 2.0 ** -24
    assert out["stop"] in (1, 2, 3)
    if out["stop"] == 1:
        assert out["nbe"][-1] <= 2.0 ** -24
    # a half bucket that holds entries at the larger epsilon
    if eps == 2.0 ** -18 and name == "convdiff3d":
        assert out["buckets"]["nnz_k"][1] > 0


def test_ir_single_working_precision_step_follows_alg31(orc):
    """One refinement step with u = fp32, u_r = fp64 equals Alg 3.1's steps
    taken one at a time: x0 = M b in u_f, stored in u; r = b - A x0 in u_r,
    stored in u; d from GMRES, stored in u; x1 = x0 + d in u."""
    wl = W.workload("convdiff3d", grid=8)
    A, P = wl["A"], wl["pattern"]
    sp_ = orc.spai(A, P, wl["spai_eps"])
    muf = orc.round_to(sp_["mval"], "fp32")
    fm = SSD["precs"]
    ids = orc.bucket_ids(P.row_ptr, muf, 2.0 ** -18, fm)["ids"]
    stored, _, _ = orc.bucket_store(P.row_ptr, P.col, muf, ids, fm)
    S = orc.System(A, P.row_ptr, P.col, stored, ids, fm)
    out = orc.gmres_ir(S, muf, wl["b"], "fp32", "fp32", 1e-4, 500, 1, u="fp32", u_r="fp64")
    r32 = lambda v: orc.round_to(v, "fp32")  # noqa: E731
    x0 = r32(orc.spmv_prec(P.row_ptr, P.col, muf, "fp32", wl["b"]))
    r = r32(orc.residual_fp64(A, x0, wl["b"]))
    d, its, _ = orc.gmres(S, r, "fp32", "fp32", 1e-4, 500)
    x1 = r32(x0 + r32(d))
    assert out["its"] == [its]
    assert np.array_equal(out["x"], x1)
    # and u = fp64 keeps the Dot2 residual and the unrounded update
    out64 = orc.gmres_ir(S, muf, wl["b"], "fp32", "fp32", 1e-4, 500, 1)
    x0 = orc.spmv_prec(P.row_ptr, P.col, muf, "fp32", wl["b"])
    d, _, _ = orc.gmres(S, orc.residual_dd(A, x0, wl["b"]), "fp32", "fp32", 1e-4, 500)
    assert np.array_equal(out64["x"], x0 + d)


def test_gmres_ir_rejects_unknown_working_precision(orc):
    wl = W.workload("convdiff2d", grid=6)
    with pytest.raises(ValueError):
        orc.solve(wl, u="fp16")


def _half_textbook_spmv(P, val, b):
    """Row sums in IEEE half with numpy's float16 type: each product and partial
    sum is one half-precision operation, columns in ascending order."""
    y = np.zeros(P.n)
    for i in range(P.n):
        acc = np.float16(0.0)
        for p in range(P.row_ptr[i], P.row_ptr[i + 1]):
            acc = np.float16(acc + np.float16(np.float16(val[p]) * np.float16(b[P.col[p]])))
        y[i] = float(acc)
    return y


def test_x0_in_half_is_the_textbook_half_product(orc):
    """(half, single, double): x0 = M b with M held in u_f = half and the
    product taken in half (Alg 3.1, first lines), then held in u = fp32."""
    wl = W.workload("convdiff2d", grid=8)
    A, P = wl["A"], wl["pattern"]
    sp_ = orc.spai(A, P, wl["spai_eps"])
    m16 = orc.round_to(sp_["mval"], "fp16")
    assert np.array_equal(m16, sp_["mval"].astype(np.float16).astype(np.float64))
    ref = _half_textbook_spmv(P, m16, wl["b"])
    assert np.array_equal(orc.spmv_prec(P.row_ptr, P.col, m16, "fp16", wl["b"]), ref)
    ids = orc.bucket_ids(P.row_ptr, m16, 2.0 ** -24, SSD["precs"])["ids"]
    stored, _, _ = orc.bucket_store(P.row_ptr, P.col, m16, ids, SSD["precs"])
    S = orc.System(A, P.row_ptr, P.col, stored, ids, SSD["precs"])
    out = orc.gmres_ir(S, m16, wl["b"], "fp32", "fp32", 1e-4, 500, 0, u="fp32", u_r="fp64", u_f="fp16")
    assert np.array_equal(out["x"], ref)
    # and the fp32 default is the same product in single
    out = orc.gmres_ir(S, m16, wl["b"], "fp32", "fp32", 1e-4, 500, 0, u="fp32", u_r="fp64")
    assert np.array_equal(out["x"], orc.spmv_prec(P.row_ptr, P.col, m16, "fp32", wl["b"]))
    assert not np.array_equal(out["x"], ref)


HSD = dict(SSD, u_f="fp16")


@pytest.mark.parametrize("name,grid", [("convdiff2d", 32), ("convdiff3d", 8)])
@pytest.mark.parametrize("eps", [2.0 ** -24, 2.0 ** -18])
def test_ir_half_single_double_reaches_single_accuracy(orc, name, grid, eps):
    """(u_f, u, u_r) = (half, single, double) (Section 4): M held in half, x0
    in half; kappa_inf(A) of these systems is far below u^-1/3 u_f^-2/3 (about
    4e4), so GMRES-IR reaches the level of u = 2^-24 as in the single setting,
    with x held in fp32."""
    wl = W.workload(name, grid=grid)
    out = orc.solve(wl, bucket_eps=eps, **HSD)
    x, xt = out["x"], wl["x_true"]
    assert np.array_equal(out["muf"], out["muf"].astype(np.float16).astype(np.float64))
    assert np.array_equal(x, x.astype(np.float32).astype(np.float64))
    assert np.abs(x - xt).max() / np.abs(xt).max() <= 2 * 2.0 ** -24
    assert out["stop"] in (1, 2, 3)
    # the half-precision M is a weaker preconditioner than the single one: never fewer
    # refinement steps than u_f = fp32 needs
    ref = orc.solve(wl, bucket_eps=eps, **SSD)
    assert out["steps"] >= ref["steps"] - 1


def test_gmres_ir_rejects_unknown_u_f(orc):
    wl = W.workload("convdiff2d", grid=6)
    with pytest.raises(ValueError):
        orc.solve(wl, u="fp32", u_r="fp64", u_f="bf16")


def test_half_product_keeps_the_half_range(orc):
    """The half product of x0 is IEEE half with its own range, as numpy's
    float16: entries and partial sums below 2^-14 become subnormal (spacing
    2^-24), products above 65504 overflow to Inf."""
    rng = np.random.default_rng(7)
    n = 40
    Ad = np.diag(rng.uniform(1, 2, n)) + np.diag(rng.uniform(-0.5, 0.5, n - 1), 1)
    P = _csr(Ad)
    vals = P.val * 2.0 ** rng.integers(-16, -6, P.nnz)  # many products in the subnormal range
    b = rng.uniform(-1, 1, n) * 2.0 ** rng.integers(-12, 2, n)
    m16 = orc.round_to(vals, "fp16")
    got = orc.spmv_prec(P.row_ptr, P.col, m16, "fp16", b)
    assert np.array_equal(got, _half_textbook_spmv(P, m16, b))
    assert np.any((np.abs(got) < 2.0 ** -14) & (got != 0))
    big = orc.round_to(P.val * 300.0, "fp16")
    got = orc.spmv_prec(P.row_ptr, P.col, big, "fp16", np.full(n, 300.0))
    with np.errstate(over="ignore"):  # the overflow is the point of this case
        ref = _half_textbook_spmv(P, big, np.full(n, 300.0))
    assert np.array_equal(np.isinf(got), np.isinf(ref)) and np.isinf(got).any()
    assert np.array_equal(got[np.isfinite(got)], ref[np.isfinite(ref)])
