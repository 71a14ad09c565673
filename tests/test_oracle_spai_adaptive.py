"""Pins for the oracle's adaptive SPAI (Alg 2.1 with alpha > 0, Grote and
Huckle's pattern growth from the identity pattern, Section 4), each against
dense linear algebra written independently of the oracle's C code:

  * one scoring pass: the shadow, the least-squares solution and residual,
    the candidate set, rho_j as the residual of the univariate minimisation
    min_mu ||sbar - mu B e_j|| (solved by LAPACK), the mean and the picks;
  * the finished M: every row is the least-squares solution on its own final
    pattern; the residual norm never grows from one pass to the next, and
    after a pass it is no larger than the smallest rho of the previous one;
  * alpha = 0 reduces to the fixed identity pattern; enough passes on a small
    matrix fill the pattern and give M = A^-1; eps large stops at once.
"""
import numpy as np
import pytest

import oracle as O
from paper_2307_03914_gb300 import workloads as W


def _dense_B(A):
    d = O.row_absmax_scale(A)
    Ad = A.to_scipy().toarray()
    return Ad.T * d[None, :], d, Ad


def _dense_pass(B, k, J, beta):
    """The same pass from dense matrices: shadow, LS, candidates, rho, picks."""
    n = B.shape[0]
    J = np.sort(np.asarray(J))
    I = np.flatnonzero(np.abs(B[:, J]).sum(axis=1) != 0)
    Ab = B[np.ix_(I, J)]
    e = (I == k).astype(float)
    m, *_ = np.linalg.lstsq(Ab, e, rcond=None)
    s = Ab @ m - e
    L = np.union1d(I, [k])
    cand = np.array([j for j in range(n) if j not in set(J) and np.any(B[L, j] != 0)], dtype=int)
    r_full = np.zeros(n)
    r_full[I] = s
    rho = []
    for j in cand:
        c = B[:, j]
        mu, *_ = np.linalg.lstsq(c[:, None], r_full, rcond=None)
        rho.append(np.linalg.norm(r_full - c * mu[0]))
    rho = np.array(rho)
    mean = rho.mean() if len(rho) else 0.0
    ok = np.flatnonzero(rho <= mean)
    order = sorted(ok, key=lambda t: (rho[t], cand[t]))
    return dict(I=I, m=m, sres=np.linalg.norm(s), cand=cand, rho=rho, mean=mean,
                picks=cand[order[:beta]])


CASES = [("random", W.random_sparse(50, 5, sigma=2.0, delta=0.4, seed=3)), ("convdiff2d", W.convdiff2d(7))]


@pytest.mark.parametrize("name,A", CASES, ids=[c[0] for c in CASES])
def test_scoring_pass_matches_dense_definitions(name, A):
    B, d, _ = _dense_B(A)
    rng = np.random.default_rng(4)
    for k in rng.choice(A.n, 6, replace=False):
        J = [int(k)]
        for _ in range(3):
            o = O.spai_score(A, int(k), J, beta=4)
            r = _dense_pass(B, int(k), J, beta=4)
            assert o["nI"] == len(r["I"])
            assert np.allclose(o["mbar"], r["m"], rtol=1e-10, atol=1e-12)
            assert o["sres"] == pytest.approx(r["sres"], rel=1e-10, abs=1e-14)
            assert np.array_equal(o["cand"], r["cand"])
            assert np.allclose(o["rho"], r["rho"], rtol=1e-9, atol=1e-12)
            assert o["mean"] == pytest.approx(r["mean"], rel=1e-10)
            assert np.array_equal(o["picks"], r["picks"]), (k, J)
            J = sorted(set(J) | set(o["picks"].tolist()))


@pytest.mark.parametrize("name,A", CASES, ids=[c[0] for c in CASES])
def test_final_rows_are_least_squares_on_their_pattern(name, A):
    B, d, _ = _dense_B(A)
    out = O.spai_adaptive(A, 0.05, alpha=3, beta=4)
    assert out["nbad"] == 0
    for k in range(A.n):
        J = out["col"][out["row_ptr"][k]:out["row_ptr"][k + 1]]
        assert np.all(np.diff(J) > 0) and k in J
        I = np.flatnonzero(np.abs(B[:, J]).sum(axis=1) != 0)
        e = (I == k).astype(float)
        m, *_ = np.linalg.lstsq(B[np.ix_(I, J)], e, rcond=None)
        got = out["mval"][out["row_ptr"][k]:out["row_ptr"][k + 1]]
        assert np.allclose(got, m * d[J], rtol=1e-9, atol=1e-13)
        assert out["resid"][k] == pytest.approx(np.linalg.norm(B[np.ix_(I, J)] @ m - e), rel=1e-9, abs=1e-14)
        steps = out["step_added"][out["row_ptr"][k]:out["row_ptr"][k + 1]]
        assert steps[list(J).index(k)] == 0
        assert steps.max() <= out["nsolves"][k] - 1
        assert out["conv"][k] == (out["resid"][k] <= 0.05)


@pytest.mark.parametrize("name,A", CASES, ids=[c[0] for c in CASES])
def test_residual_decreases_and_stays_below_best_rho(name, A):
    """The LS residual on J u picks is no larger than the univariate residual
    along the best pick (min rho), which is no larger than ||sbar|| itself."""
    for k in range(0, A.n, 5):
        J = [k]
        prev = None
        for _ in range(4):
            o = O.spai_score(A, k, J, beta=8)
            if prev is not None:
                assert o["sres"] <= prev["sres"] * (1 + 1e-12) + 1e-15
                assert o["sres"] <= prev["rho"].min() * (1 + 1e-12) + 1e-15
            if len(o["picks"]) == 0:
                break
            assert o["rho"].min() <= o["sres"] * (1 + 1e-12)
            prev = o
            J = sorted(set(J) | set(o["picks"].tolist()))


def test_alpha_zero_is_the_fixed_identity_pattern():
    A = W.random_sparse(60, 6, sigma=1.5, delta=0.4, seed=8)
    out = O.spai_adaptive(A, 0.1, alpha=0)
    P = W.CSR(A.n, np.arange(A.n + 1, dtype=np.int32), np.arange(A.n, dtype=np.int32), np.ones(A.n))
    fixed = O.spai(A, P, 0.1)
    assert np.array_equal(out["col"], np.arange(A.n))
    assert np.allclose(out["mval"], fixed["mval"], rtol=1e-14, atol=0)
    assert np.allclose(out["resid"], fixed["resid"], rtol=1e-14, atol=0)
    assert np.all(out["nsolves"] == 1)


def test_growth_fills_a_small_matrix_to_the_inverse():
    """With enough passes and a tolerance no column meets early, the pattern
    grows to every index that can reduce the residual; on a small nonsingular
    matrix whose inverse is dense this ends at M = A^-1."""
    A = W.convdiff2d(4)
    Ainv = np.linalg.inv(A.to_scipy().toarray())
    out = O.spai_adaptive(A, 1e-13, alpha=12, beta=8, cap=A.n)
    Md = np.zeros((A.n, A.n))
    for k in range(A.n):
        sl = slice(out["row_ptr"][k], out["row_ptr"][k + 1])
        Md[k, out["col"][sl]] = out["mval"][sl]
    assert np.abs(Md - Ainv).max() <= 1e-10 * np.abs(Ainv).max()
    assert out["conv"].all()


def test_large_tolerance_stops_after_the_first_solve():
    A = W.convdiff2d(6)
    out = O.spai_adaptive(A, 10.0, alpha=3)
    assert np.all(out["nsolves"] == 1) and np.all(out["nJ"] == 1) and out["conv"].all()


def test_shadow_cap_stops_growth_and_keeps_the_last_solution():
    A = W.random_sparse(80, 9, sigma=2.0, delta=0.4, seed=12)
    full = O.spai_adaptive(A, 1e-6, alpha=3, beta=8, imax_rows=10 ** 6)
    capped = O.spai_adaptive(A, 1e-6, alpha=3, beta=8, imax_rows=20)
    assert capped["capped"].sum() > 0
    B, d, _ = _dense_B(A)
    for k in np.flatnonzero(capped["capped"]):
        J = capped["col"][capped["row_ptr"][k]:capped["row_ptr"][k + 1]]
        I = np.flatnonzero(np.abs(B[:, J]).sum(axis=1) != 0)
        assert len(I) <= 20
        assert capped["nJ"][k] <= full["nJ"][k]
