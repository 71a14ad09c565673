"""Pins for the oracle's fixed-pattern SPAI (eq. fronormmin, eq. redprob,
Alg 2.1 with alpha = 0, column scaling of Section 4, Alg 3.1 first line).

Independent checks: LAPACK least squares (numpy.linalg.lstsq) on blocks cut
out with scipy, M = A^-1 for a full pattern, and the Frobenius-norm
decoupling ||I - M A||_F^2 = sum_k ||sbar_k||^2 (which also fixes the
orientation M = M'^T D of a left preconditioner).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2307_03914_gb300 import workloads as W


@pytest.mark.parametrize("m,k", [(1, 1), (5, 5), (13, 5), (25, 7), (60, 24), (400, 24)])
def test_householder_ls_vs_lapack(orc, m, k):
    rng = np.random.default_rng(m * 100 + k)
    A = rng.normal(size=(m, k))
    b = rng.normal(size=m)
    x, res, rd = orc.householder_ls(A, b)
    ref, *_ = np.linalg.lstsq(A, b, rcond=None)
    assert rd == 0
    assert np.linalg.norm(x - ref) <= 1e-12 * max(1.0, np.linalg.norm(ref)) * np.linalg.cond(A)
    assert abs(res - np.linalg.norm(A @ ref - b)) <= 1e-12 * max(1.0, np.linalg.norm(b))


def test_householder_flags_rank_deficiency(orc):
    A = np.array([[1.0, 2.0], [2.0, 4.0], [3.0, 6.0]])
    x, _, rd = orc.householder_ls(A, np.ones(3), rank_tol=1e-12)
    assert rd == 1 and np.all(x == 0)


def _blocks(A, P, d, k):
    """Abar and ebar of column k cut out of B = A^T D with scipy (eq. redprob)."""
    B = (A.to_scipy().T @ sp.diags(d)).tocsc()
    J = P.col[P.row_ptr[k]:P.row_ptr[k + 1]]
    sub = B[:, J]
    I = np.unique(sub.nonzero()[0])
    Ab = sub[I, :].toarray()
    e = (I == k).astype(float)
    return Ab, e, J


@pytest.mark.parametrize("name", ["convdiff2d", "convdiff3d", "random"])
def test_spai_columns_vs_lapack(orc, name):
    if name == "convdiff2d":
        A = W.convdiff2d(12)
        P = W.pattern_of(A)
    elif name == "convdiff3d":
        A = W.convdiff3d(6)
        P = W.pattern_of(A)
    else:
        A = W.random_sparse(300, 8, seed=5)
        P = W.pattern_power_topk(A, 12)
    out = orc.spai(A, P, 0.3)
    d = orc.row_absmax_scale(A)
    rng = np.random.default_rng(0)
    for k in rng.choice(A.n, size=min(40, A.n), replace=False):
        Ab, e, J = _blocks(A, P, d, k)
        ref, *_ = np.linalg.lstsq(Ab, e, rcond=None)
        mrow = out["mval"][P.row_ptr[k]:P.row_ptr[k + 1]]
        mbar = mrow / d[J]  # undo M = M'^T D
        assert np.allclose(mbar, ref, rtol=1e-11, atol=1e-13), k
        # normal equations of the least-squares problem
        s = Ab @ mbar - e
        assert np.linalg.norm(Ab.T @ s) <= 1e-12 * np.linalg.norm(Ab) * max(np.linalg.norm(s), 1e-300) + 1e-14
        assert abs(out["resid"][k] - np.linalg.norm(s)) <= 1e-12
        assert out["conv"][k] == (out["resid"][k] <= 0.3)
        # an optimal solution: random perturbations never reduce the residual
        for _ in range(5):
            dlt = rng.normal(size=mbar.size) * 1e-3
            assert np.linalg.norm(Ab @ (mbar + dlt) - e) >= np.linalg.norm(s) - 1e-15


def test_full_pattern_gives_inverse(orc):
    rng = np.random.default_rng(11)
    n = 12
    Ad = rng.normal(size=(n, n)) + 6 * np.eye(n)
    Asp = sp.csr_matrix(Ad)
    A = W.CSR(n, Asp.indptr.astype(np.int32), Asp.indices.astype(np.int32), Asp.data.astype(float))
    P = W.pattern_of(A)  # dense pattern
    out = orc.spai(A, P, 0.1)
    M = sp.csr_matrix((out["mval"], P.col, P.row_ptr), shape=(n, n)).toarray()
    assert np.allclose(M, np.linalg.inv(Ad), rtol=1e-12, atol=1e-12)
    assert np.all(out["resid"] < 1e-12)


def test_frobenius_decoupling_and_orientation(orc):
    A = W.convdiff2d(10)
    P = W.pattern_of(A)
    out = orc.spai(A, P, 0.3)
    M = sp.csr_matrix((out["mval"], P.col, P.row_ptr), shape=(A.n, A.n))
    lhs = np.linalg.norm(np.eye(A.n) - (M @ A.to_scipy()).toarray(), "fro") ** 2
    assert abs(lhs - np.sum(out["resid"] ** 2)) <= 1e-10 * lhs
    # the transposed reading (right preconditioner) does not satisfy it
    bad = np.linalg.norm(np.eye(A.n) - (A.to_scipy() @ M).toarray(), "fro") ** 2
    assert abs(bad - lhs) > 1e-6 * lhs


def test_scaling_normalises_columns_of_AT(orc):
    A = W.random_sparse(200, 8, seed=3)
    d = orc.row_absmax_scale(A)
    B = abs(A.to_scipy().T @ sp.diags(d)).tocsc()
    colmax = B.max(axis=0).toarray().ravel()
    assert np.all(np.abs(colmax - 1.0) <= 2.0 ** -52)
