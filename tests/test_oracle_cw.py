"""Pins for the oracle's componentwise (x-dependent) bucketing, the strategy
of Graillat et al. that Section 2.3 mentions and sets aside because the buckets
depend on the vector x.  The paper does not print the rule; the reading used
here is eq. (nint) applied row by row to the products |a_ij| |x_j| against
eps (|A||x|)_i / u_k.  What pins it:

  * the componentwise backward error of the bucketed product,
    max_i |yhat_i - y_i| / (|A||x|)_i, stays within (q - 1) u_1 + c eps with
    c from eq. (ccw) -- checked with exact rationals, in both the literal
    (partial sums in u_k) and the decoupled (fp32 / fp64 accumulation) forms;
  * with x = 1 the rule is eq. (nint) with ||A|| replaced by the row's sum of
    |a_ij|, so on the rows that attain ||A||_inf it gives the normwise
    bucketing's ids (an independent routine);
  * powers of two leave it unchanged: x scaled as a whole, or one row of A;
  * a row with a single entry lands where a 1 x 1 matrix does under the
    normwise rule; q = 1 puts everything in bucket 1; the buckets partition
    the nonzeros.
"""
from fractions import Fraction

import numpy as np

from paper_2307_03914_gb300 import workloads as W

FMTS = ["fp64", "fp32", "bf16", "drop"]
US = [2.0 ** -53, 2.0 ** -24, 2.0 ** -8, 1.0]


def _exact_rows(A, vals, x):
    y, ax = [], []
    for i in range(A.n):
        ps = range(A.row_ptr[i], A.row_ptr[i + 1])
        y.append(sum((Fraction(vals[p]) * Fraction(x[A.col[p]]) for p in ps), Fraction(0)))
        ax.append(sum((abs(Fraction(vals[p]) * Fraction(x[A.col[p]])) for p in ps), Fraction(0)))
    return y, ax


def test_cw_bucketing_meets_componentwise_bound(orc):
    rng = np.random.default_rng(31)
    q = len(FMTS)
    for trial in range(5):
        A = W.random_sparse(50, 9, sigma=3.0, seed=60 + trial)
        vals = A.val * np.exp(rng.normal(0, 4, A.nnz))
        x = rng.uniform(-1, 1, A.n) * np.exp(rng.normal(0, 3, A.n))
        yex, ax = _exact_rows(A, vals, x)
        for eps in [2.0 ** -40, 2.0 ** -24, 2.0 ** -12, 2.0 ** -6]:
            bk = orc.bucket_ids_cw(A.row_ptr, A.col, vals, x, eps, FMTS)
            assert bk["nnz_k"].sum() == A.nnz
            p = np.zeros((A.n, q))
            for i in range(A.n):
                p[i] = np.bincount(bk["ids"][A.row_ptr[i]:A.row_ptr[i + 1]], minlength=q)
            c = (1 + (q - 1) * US[0]) + np.max((p ** 2 * (1 + np.array(US)) ** 2).sum(axis=1))
            bound = (q - 1) * US[0] + c * eps
            stored, _, _ = orc.bucket_store(A.row_ptr, A.col, vals, bk["ids"], FMTS)
            for y in (orc.bspmv_literal(A.row_ptr, A.col, vals, bk["ids"], FMTS, x),
                      orc.bspmv(A.row_ptr, A.col, stored, bk["ids"], FMTS, x)):
                ecw = max(float(abs(Fraction(y[i]) - yex[i]) / ax[i]) for i in range(A.n) if ax[i] > 0)
                assert ecw <= bound, (trial, eps, ecw, bound)


def test_cw_with_unit_x_is_normwise_on_max_rows(orc):
    rng = np.random.default_rng(5)
    for trial in range(4):
        A = W.random_sparse(64, 7, sigma=2.0, seed=90 + trial)
        vals = A.val.copy()
        # make several rows attain ||A||_inf exactly (rows scaled to the same abs sum)
        rs = np.array([np.abs(vals[A.row_ptr[i]:A.row_ptr[i + 1]]).sum() for i in range(A.n)])
        top = rng.choice(A.n, 8, replace=False)
        for i in top:
            sl = slice(A.row_ptr[i], A.row_ptr[i + 1])
            vals[sl] = vals[sl] * (2.0 ** np.ceil(np.log2(rs.max() * 4 / rs[i])))
        for eps in [2.0 ** -30, 2.0 ** -14, 2.0 ** -7]:
            cw = orc.bucket_ids_cw(A.row_ptr, A.col, vals, np.ones(A.n), eps, FMTS)
            nw = orc.bucket_ids(A.row_ptr, vals, eps, FMTS)
            for i in range(A.n):
                sl = slice(A.row_ptr[i], A.row_ptr[i + 1])
                if cw["srow"][i] == nw["norm"]:
                    assert np.array_equal(cw["ids"][sl], nw["ids"][sl]), (trial, eps, i)
            assert any(cw["srow"][i] == nw["norm"] for i in range(A.n))


def test_cw_power_of_two_invariance_and_special_cases(orc):
    rng = np.random.default_rng(11)
    A = W.random_sparse(70, 8, sigma=2.5, seed=123)
    x = rng.uniform(-1, 1, A.n)
    eps = 2.0 ** -16
    base = orc.bucket_ids_cw(A.row_ptr, A.col, A.val, x, eps, FMTS)["ids"]
    assert np.array_equal(orc.bucket_ids_cw(A.row_ptr, A.col, A.val, x * 2.0 ** 37, eps, FMTS)["ids"], base)
    vals = A.val.copy()
    i = 17
    vals[A.row_ptr[i]:A.row_ptr[i + 1]] *= 2.0 ** -29
    assert np.array_equal(orc.bucket_ids_cw(A.row_ptr, A.col, vals, x, eps, FMTS)["ids"], base)
    one = orc.bucket_ids_cw(A.row_ptr, A.col, A.val, x, eps, ["fp64"])
    assert np.all(one["ids"] == 0) and one["nnz_k"][0] == A.nnz
    # a single entry per row (a diagonal matrix) is its row's whole |A||x|: the
    # bucket k with eps / u_(k+1) < 1 <= eps / u_k, as for a 1 x 1 normwise case
    D = W.CSR(5, np.arange(6), np.arange(5), np.array([3.0, -1e-9, 7e5, 2.0 ** -60, 1.0]))
    xd = np.array([1e-3, 2.0, -5.0, 1e10, 1.0])
    for eps, k in [(2.0 ** -30, 0), (2.0 ** -20, 1), (2.0 ** -5, 2)]:
        ids = orc.bucket_ids_cw(D.row_ptr, D.col, D.val, xd, eps, FMTS)["ids"]
        assert np.all(ids == k), (eps, ids)
        assert orc.bucket_ids(np.array([0, 1]), np.array([0.37]), eps, FMTS)["ids"][0] == k
