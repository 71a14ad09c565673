"""GPU parity of the (u_f, u, u_r) = (half, single, double) setting (Section 4):
the SPAI computed in u_f = half (every operation of the least-squares solve an
IEEE half operation, with the column scaling of Section 4 guarding the range),
M held in half, x0 = M b in half (Alg 3.1), then u = fp32 refinement with the
residual in fp64 and buckets {single, half, drop}.

Bars:
  * M imported in half (values rounded once from fp64) and x0 = M b in half:
    bit-exact against the oracle;
  * the GPU's half SPAI against the oracle's fp64 SPAI: per column the
    first-order least-squares perturbation bound with u_f = 2^-11, every entry
    a half value; column residuals within the rounding error of s = Abar m - e
    taken in half, (|J| + 2) u_f (||(|M| |A|)(k, :)||_2 + 1), plus the
    second-order change that the perturbation of m makes to the optimal
    residual;
  * refinement: x is fp32-valued; both sides reach forward error <= 2u
    (u = 2^-24) and agree within 4u; refinement steps within one.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle as O
from gpu_helpers import dev, gpu_bucket, host, lib, small_workloads, spai_tolerance
from paper_2307_03914_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# the convection-diffusion cases (|I| <= 33 rows per block).  The random case
# has blocks of about 300 rows, where the rank test |R_jj| <= |I| u_f ||Abar||_F
# becomes 0.15 ||Abar||_F in half and flags most columns; it is checked for
# those flags only.
ALL = small_workloads()
WLS = [w for w in ALL if w["name"] != "random"]
RANDOM = [w for w in ALL if w["name"] == "random"][0]
IDS = [f"{w['name']}-{w['A'].n}" for w in WLS]
U = 2.0 ** -24
UF = 2.0 ** -11
PRECS = ["fp32", "fp16", "drop"]


@pytest.fixture(scope="module")
def B():
    return lib()


def _half_build(B, wl):
    A = B.DeviceCSR.from_host(wl["A"])
    P = B.DeviceCSR.from_host(wl["pattern"], with_values=False)
    M, info = B.bspai_build(A, P, wl["spai_eps"], u_f="fp16")
    n, nnz = wl["A"].n, wl["pattern"].nnz
    _, _, v, res = B.M_export(M, n, nnz)
    return dict(A=A, M=M, info=info, val=host(v).astype(np.float64), resid=host(res).astype(np.float64))


def _oracle_half_M(B, wl):
    """The oracle's SPAI handed to the library in u_f = half (rounded there once
    from fp64), with the oracle's own half values."""
    P = wl["pattern"]
    ref = O.spai(wl["A"], P, wl["spai_eps"], u_f=UF)
    Md = B.DeviceCSR(P.n, dev(P.row_ptr.astype(np.int32)), dev(P.col.astype(np.int32)), dev(ref["mval"]))
    return B.M_create(Md, u_f="fp16"), O.round_to(ref["mval"], "fp16")


@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_M_create_half_rounds_once(B, wl):
    P = wl["pattern"]
    M, m16 = _oracle_half_M(B, wl)
    _, _, v, _ = B.M_export(M, P.n, P.nnz)
    assert np.array_equal(host(v).astype(np.float64), m16)


@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_x0_in_half_bitexact(B, wl):
    P = wl["pattern"]
    M, m16 = _oracle_half_M(B, wl)
    y = torch.empty(P.n, dtype=torch.float64, device="cuda")
    B.apply_uf(M, dev(wl["b"]), y)
    ref = O.spmv_prec(P.row_ptr, P.col, m16, "fp16", wl["b"])
    assert np.array_equal(host(y), ref)
    # a random x with entries across several binades
    x = np.random.default_rng(41).uniform(-1, 1, P.n) * 2.0 ** np.random.default_rng(42).integers(-8, 8, P.n)
    B.apply_uf(M, dev(x), y)
    assert np.array_equal(host(y), O.spmv_prec(P.row_ptr, P.col, m16, "fp16", x))


@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_half_spai_within_perturbation_bound(B, wl):
    A, P = wl["A"], wl["pattern"]
    g = _half_build(B, wl)
    assert g["info"]["status"] == 0 and g["info"]["n_rank_deficient"] == 0
    assert np.array_equal(g["val"], O.round_to(g["val"], "fp16"))
    ref = O.spai(A, P, wl["spai_eps"], u_f=UF)
    tol = spai_tolerance(ref["kappa"], ref["resid"], UF)
    worst = 0.0
    for k in range(A.n):
        a, b = P.row_ptr[k], P.row_ptr[k + 1]
        e = np.linalg.norm(g["val"][a:b] - ref["mval"][a:b]) / np.linalg.norm(ref["mval"][a:b])
        worst = max(worst, e / tol[k])
        assert e <= tol[k], (k, e, tol[k])
    # w_k = ||(|M| |A|)(k, :)||_2 = || |Abar| |mbar| ||_2 (B = A^T D, m = M(k, J) / d_J)
    Ms = sp.csr_matrix((np.abs(ref["mval"]), P.col, P.row_ptr), shape=(A.n, A.n))
    As = sp.csr_matrix((np.abs(A.val), A.col, A.row_ptr), shape=(A.n, A.n))
    w = np.sqrt(np.asarray((Ms @ As).multiply(Ms @ As).sum(axis=1)).ravel())
    nJ = np.diff(P.row_ptr)
    bar = 2 * (nJ + 2) * UF * (w + 1) + (tol * w) ** 2 / (2 * np.maximum(ref["resid"], 1e-3))
    assert np.all(np.abs(g["resid"] - ref["resid"]) <= bar), np.max(np.abs(g["resid"] - ref["resid"]) / bar)
    clear = np.abs(ref["resid"] - wl["spai_eps"]) > bar
    assert np.array_equal((g["resid"] <= wl["spai_eps"])[clear], (ref["conv"] == 1)[clear])
    print(f"{wl['name']}: worst half SPAI error / tolerance = {worst:.3f}")


def _check(info, xg, ref, wl):
    xt = wl["x_true"]
    assert info["status"] == 0, info
    assert np.array_equal(xg, xg.astype(np.float32).astype(np.float64))
    fe_g = np.abs(xg - xt).max() / np.abs(xt).max()
    fe_o = np.abs(ref["x"] - xt).max() / np.abs(xt).max()
    assert fe_g <= 2 * U and fe_o <= 2 * U, (fe_g, fe_o)
    assert np.abs(xg - ref["x"]).max() <= 4 * U * np.abs(ref["x"]).max()
    assert abs(info["ir_steps"] - ref["steps"]) <= 1


@pytest.mark.parametrize("eps", [2.0 ** -24, 2.0 ** -18])
@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_ir_half_single_double_matches_oracle(B, wl, eps):
    """The whole setting on the GPU (half SPAI built there) against the oracle's
    pipeline with M rounded to half."""
    A, P = wl["A"], wl["pattern"]
    g = _half_build(B, wl)
    bm = gpu_bucket(B, g["M"], P.nnz, eps, PRECS)
    x = torch.empty(A.n, dtype=torch.float64, device="cuda")
    info = B.gmres_ir_solve(g["A"], dev(wl["b"]), bm["BM"], g["M"], x, u="fp32", u_r="fp64", u_g="fp32",
                            u_p="fp32", tol=1e-4)
    ref = O.solve(wl, bucket_eps=eps, precs=PRECS, u="fp32", u_r="fp64", ug="fp32", up="fp32", tau=1e-4,
                  u_f="fp16")
    _check(info, host(x), ref, wl)


@pytest.mark.parametrize("wl", WLS[:3], ids=IDS[:3])
def test_ir_half_on_oracle_M_matches_oracle(B, wl):
    """The oracle's half M handed to the library: x0 and the buckets are then
    the oracle's to the bit, and the refinement counts agree as in the single
    setting (first GMRES count within max(2, 10 %))."""
    A, P = wl["A"], wl["pattern"]
    eps = 2.0 ** -18
    M, m16 = _oracle_half_M(B, wl)
    bm = gpu_bucket(B, M, P.nnz, eps, PRECS)
    ref = O.solve(wl, bucket_eps=eps, precs=PRECS, u="fp32", u_r="fp64", ug="fp32", up="fp32", tau=1e-4,
                  u_f="fp16")
    assert np.array_equal(bm["ids"], ref["buckets"]["ids"])
    Ah = B.matrix_create(B.DeviceCSR.from_host(A))
    x = torch.empty(A.n, dtype=torch.float64, device="cuda")
    info = B.gmres_ir_solve(Ah, dev(wl["b"]), bm["BM"], M, x, u="fp32", u_r="fp64", u_g="fp32", u_p="fp32",
                            tol=1e-4)
    _check(info, host(x), ref, wl)
    assert abs(info["gmres_iters"][0] - ref["its"][0]) <= max(2, 0.1 * ref["its"][0])


def test_half_spai_rank_test_on_wide_blocks(B):
    """With |I| of about 300 rows the rank test |R_jj| <= |I| u_f ||Abar||_F
    flags most blocks in half although they are well conditioned (kappa of
    about 27): the tolerance is 0.15 ||Abar||_F.  The oracle applies the same
    test and flags them too.  Flagged columns of M are zero."""
    wl = RANDOM
    P = wl["pattern"]
    A = B.DeviceCSR.from_host(wl["A"])
    Pd = B.DeviceCSR.from_host(P, with_values=False)
    M, info = B.bspai_build(A, Pd, wl["spai_eps"], u_f="fp16")
    ref = O.spai(wl["A"], P, wl["spai_eps"], u_f=UF)
    assert info["status"] == B.RANK_DEFICIENT and info["n_rank_deficient"] > 0 and ref["rankdef"].sum() > 0
    _, _, v, res = B.M_export(M, P.n, P.nnz)
    v, res = host(v), host(res)
    zero_rows = [k for k in range(P.n) if not np.any(v[P.row_ptr[k]:P.row_ptr[k + 1]])]
    assert len(zero_rows) == info["n_rank_deficient"]
    assert np.all(res[zero_rows] == 1.0)
    print(f"rank-deficient blocks in half: GPU {info['n_rank_deficient']}, oracle {int(ref['rankdef'].sum())}")


def test_half_u_f_only_fp16_or_fp32(B):
    wl = WLS[0]
    A = B.DeviceCSR.from_host(wl["A"])
    P = B.DeviceCSR.from_host(wl["pattern"], with_values=False)
    with pytest.raises(Exception):
        B.bspai_build(A, P, wl["spai_eps"], u_f="bf16")
    with pytest.raises(Exception):
        B.M_create(B.DeviceCSR.from_host(wl["A"]), u_f="e4m3")


# ---------------------------------------------------------------- adaptive SPAI in half
# A rho computed in half differs from the oracle's fp64 rho by the rounding of
# its half reductions, up to about |I| u_f relative with |I| <= 64 rows here:
# picks may differ where two values lie within that of each other.
TIE_H = 64 * UF


def _near_tie_h(o, j, picks_other):
    rho = dict(zip(o["cand"].tolist(), o["rho"].tolist()))
    if j not in rho:
        return False
    ends = [o["mean"]]
    for p in (o["picks"].tolist(), picks_other):
        vals = [rho[x] for x in p if x in rho]
        if vals:
            ends.append(max(vals))
    return any(abs(rho[j] - t) <= TIE_H * max(abs(t), 1e-30) for t in ends)


@pytest.mark.parametrize("eps,alpha", [(0.3, 3), (0.1, 2)])
@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_adaptive_half_spai_matches_oracle(B, wl, eps, alpha):
    """Alg 2.1 with alpha > 0 from the identity pattern, every operation in
    half: each pass the GPU took is replayed with the oracle's fp64 scoring on
    the GPU's own pattern (same picks, or a difference only at a near tie
    within TIE_H); the final values are the least-squares solution on the
    GPU's final pattern within the half perturbation bound."""
    A = wl["A"]
    n = A.n
    M, info = B.bspai_build_adaptive(B.DeviceCSR.from_host(A), eps, alpha, 8, 256, u_f="fp16")
    assert info["status"] == 0 and info["n_rank_deficient"] == 0
    nnz = int(info["nnz"])
    rp, ci, v, res = B.M_export(M, n, nnz)
    step, cinfo = B.M_adaptive_export(M, n, nnz)
    rp, ci, val, resid = host(rp), host(ci), host(v).astype(np.float64), host(res).astype(np.float64)
    step, cinfo = host(step).astype(int), host(cinfo)
    assert np.array_equal(val, O.round_to(val, "fp16"))
    ref = O.spai_adaptive(A, eps, alpha, beta=8, imax_rows=256, u_f=UF)
    differ = ties = 0
    for k in range(n):
        J, st = ci[rp[k]:rp[k + 1]], step[rp[k]:rp[k + 1]]
        assert np.all(np.diff(J) > 0) and k in J
        if not np.array_equal(J, ref["col"][ref["row_ptr"][k]:ref["row_ptr"][k + 1]]):
            differ += 1
        Js = [k]
        for s in range(1, int(st.max()) + 1):
            added = sorted(J[st == s].tolist())
            o = O.spai_score(A, k, Js, beta=8, u_f=UF)
            mine = sorted(o["picks"].tolist())
            if added != mine:
                for j in set(added) ^ set(mine):
                    assert _near_tie_h(o, j, added), (k, s, added, mine)
                ties += 1
            Js = sorted(set(Js) | set(added))
    P = W.CSR(n, rp, ci, np.ones(len(ci)))
    fx = O.spai(A, P, eps, u_f=UF)
    tol = spai_tolerance(fx["kappa"], fx["resid"], UF)
    for k in range(n):
        a, b = rp[k], rp[k + 1]
        e = np.linalg.norm(val[a:b] - fx["mval"][a:b]) / np.linalg.norm(fx["mval"][a:b])
        assert e <= tol[k], (k, e, tol[k])
    Ms = sp.csr_matrix((np.abs(fx["mval"]), ci, rp), shape=(n, n))
    As = sp.csr_matrix((np.abs(A.val), A.col, A.row_ptr), shape=(n, n))
    w = np.sqrt(np.asarray((Ms @ As).multiply(Ms @ As).sum(axis=1)).ravel())
    bar = 2 * (np.diff(rp) + 2) * UF * (w + 1) + (tol * w) ** 2 / (2 * np.maximum(fx["resid"], 1e-3))
    assert np.all(np.abs(resid - fx["resid"]) <= bar)
    conv = (cinfo >> 8) & 1
    clear = np.abs(fx["resid"] - eps) > bar
    assert np.array_equal(conv[clear] == 1, (resid <= eps)[clear])
    assert info["n_converged"] == int(conv.sum())
    assert differ <= max(3, 0.1 * n), (differ, ties)
    print(f"{wl['name']} eps={eps} alpha={alpha} half: {differ} columns differ, {ties} near-tie passes")


@pytest.mark.parametrize("wl", WLS[:3], ids=IDS[:3])
def test_ir_half_adaptive_matches_oracle(B, wl):
    """The paper's (half, single, double) configuration: adaptive SPAI from the
    identity (beta = 8) in half, M in half, u = fp32, u_r = fp64."""
    A, P = wl["A"], wl["pattern"]
    eps = 2.0 ** -18
    ad = dict(spai_eps=0.3, alpha=3, beta=8)
    M, info = B.bspai_build_adaptive(B.DeviceCSR.from_host(A), ad["spai_eps"], ad["alpha"], ad["beta"], 256,
                                     u_f="fp16")
    bm = gpu_bucket(B, M, int(info["nnz"]), eps, PRECS)
    Ah = B.matrix_create(B.DeviceCSR.from_host(A))
    x = torch.empty(A.n, dtype=torch.float64, device="cuda")
    sinfo = B.gmres_ir_solve(Ah, dev(wl["b"]), bm["BM"], M, x, u="fp32", u_r="fp64", u_g="fp32", u_p="fp32",
                             tol=1e-4)
    ref = O.solve(wl, bucket_eps=eps, precs=PRECS, u="fp32", u_r="fp64", ug="fp32", up="fp32", tau=1e-4,
                  u_f="fp16", adaptive=dict(ad, u_f=UF))
    _check(sinfo, host(x), ref, wl)


# ---------------------------------------------------------------- edge cases
def test_half_M_overflow_reported(B):
    """A scaled by 2^-20: Section 4's scaling makes B = A^T D the same matrix,
    so mbar is unchanged and M = M'^T D grows by exactly 2^20.  In fp32 that
    is M's unscaled values times 2^20, to the bit; in half the entries leave
    the range (the oracle's half rounding gives Inf there too) and both builds
    report BSPAI_NONFINITE."""
    wl = WLS[0]
    A, P = wl["A"], wl["pattern"]
    As = W.CSR(A.n, A.row_ptr, A.col, A.val * 2.0 ** -20)
    Pd = B.DeviceCSR.from_host(P, with_values=False)
    M1, i1 = B.bspai_build(B.DeviceCSR.from_host(A), Pd, wl["spai_eps"])
    M2, i2 = B.bspai_build(B.DeviceCSR.from_host(As), Pd, wl["spai_eps"])
    v1 = host(B.M_export(M1, A.n, P.nnz)[2]).astype(np.float64)
    v2 = host(B.M_export(M2, A.n, P.nnz)[2]).astype(np.float64)
    assert i1["status"] == i2["status"] == 0 and np.array_equal(v2, v1 * 2.0 ** 20)
    ref = O.spai(As, P, wl["spai_eps"], u_f=UF)
    assert np.isinf(O.round_to(ref["mval"], "fp16")).any()
    with pytest.raises(B.BspaiError) as e:
        B.bspai_build(B.DeviceCSR.from_host(As), Pd, wl["spai_eps"], u_f="fp16")
    assert e.value.status == B.NONFINITE
    with pytest.raises(B.BspaiError) as e:
        B.bspai_build_adaptive(B.DeviceCSR.from_host(As), 0.3, 2, 8, 256, u_f="fp16")
    assert e.value.status == B.NONFINITE
    # and the library is still usable
    M3, i3 = B.bspai_build(B.DeviceCSR.from_host(A), Pd, wl["spai_eps"], u_f="fp16")
    assert i3["status"] == 0


@pytest.mark.parametrize("n", [1, 2, 31, 33, 65])
def test_half_ragged_1d(B, n):
    """Tiny and ragged orders (one partial 32-row slice, or a full one plus a
    tail) through the whole half setting."""
    A = W.convdiff2d(n, 1, (0.5, 0.0))
    x_true, b = W.rhs(A)
    wl = dict(name="edge", A=A, pattern=W.pattern_of(A), x_true=x_true, b=b, spai_eps=0.3,
              precs=PRECS, tau=1e-4, bucket_eps=2.0 ** -18, u_g="fp32", u_p="fp32")
    g = _half_build(B, wl)
    bm = gpu_bucket(B, g["M"], wl["pattern"].nnz, 2.0 ** -18, PRECS)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    info = B.gmres_ir_solve(g["A"], dev(b), bm["BM"], g["M"], x, u="fp32", u_r="fp64", u_g="fp32", u_p="fp32",
                            tol=1e-4)
    ref = O.solve(wl, bucket_eps=2.0 ** -18, precs=PRECS, u="fp32", u_r="fp64", ug="fp32", up="fp32", tau=1e-4,
                  u_f="fp16")
    _check(info, host(x), ref, wl)
    # b = 0 gives x = 0
    x0 = torch.empty(n, dtype=torch.float64, device="cuda")
    info = B.gmres_ir_solve(g["A"], dev(np.zeros(n)), bm["BM"], g["M"], x0, u="fp32", u_r="fp64", u_g="fp32",
                            u_p="fp32", tol=1e-4)
    assert info["status"] == 0 and torch.all(x0 == 0)
