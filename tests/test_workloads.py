"""Checks on the seeded synthetic inputs (shapes and structure of the
workloads; no method arithmetic)."""
import numpy as np

from paper_2307_03914_gb300 import workloads as W


def test_convdiff2d_size():
    A = W.convdiff2d(32)
    assert A.n == 1024 and A.nnz == 4992
    assert np.all(np.diff(A.col[A.row_ptr[0]:A.row_ptr[1]]) > 0)


def test_convdiff3d_size_formula():
    for g in (4, 7, 16):
        A = W.convdiff3d(g)
        assert A.n == g ** 3 and A.nnz == 7 * g ** 3 - 6 * g ** 2
    # 128^3 gives the 14,581,760 nonzeros of the large workload
    assert 7 * 128 ** 3 - 6 * 128 ** 2 == 14_581_760


def test_random_sparse_structure():
    A = W.random_sparse(2000, 16, seed=3)
    L = np.diff(A.row_ptr)
    assert np.all(L == 17)
    for i in range(0, 2000, 97):
        c = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0) and i in c
        v = A.val[A.row_ptr[i]:A.row_ptr[i + 1]]
        off = np.abs(v[c != i]).sum()
        assert v[c == i][0] > off  # strictly diagonally dominant
    B = W.random_sparse(2000, 16, seed=3)
    assert np.array_equal(A.val, B.val)  # seeded


def test_pattern_power_topk():
    A = W.random_sparse(500, 16, seed=4)
    P = W.pattern_power_topk(A, 24)
    assert np.all(np.diff(P.row_ptr) == 24)
    S = abs(A.to_scipy())
    C = (S @ S).toarray()
    for k in range(0, 500, 37):
        cols = P.col[P.row_ptr[k]:P.row_ptr[k + 1]]
        assert k in cols and np.all(np.diff(cols) > 0)
        row = C[k].copy()
        row[k] = np.inf
        thresh = np.sort(row)[::-1][23]
        assert np.all(row[cols] >= thresh)


def test_rhs_seeded():
    A = W.convdiff2d(8)
    x1, b1 = W.rhs(A, seed=1)
    x2, b2 = W.rhs(A, seed=1)
    assert np.array_equal(b1, b2) and np.abs(x1).max() <= 1
    assert np.allclose(A.to_scipy() @ x1, b1)
