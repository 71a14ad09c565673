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


def test_random_workload_conditioning_recorded():
    """The random workload's diagonal factor is the one the recorded search
    found (oracle/condition_random.py), whose Hager-Higham estimate of
    kappa_inf(A) at n = 65,536 lies in the target [5e5, 2e6]."""
    import json
    import os

    rec = json.load(open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                                      "random_conditioning.json")))
    assert rec["n"] == 65536 and rec["delta"] == W.RANDOM_DELTA
    assert rec["target"][0] <= rec["kappa_inf_estimate"] <= rec["target"][1]
    wl = W.workload("random", n=512)
    A = wl["A"]
    for i in range(0, A.n, 37):
        lo, hi = A.row_ptr[i], A.row_ptr[i + 1]
        diag = [A.val[p] for p in range(lo, hi) if A.col[p] == i][0]
        off = sum(abs(A.val[p]) for p in range(lo, hi) if A.col[p] != i)
        assert abs(diag - (1 + W.RANDOM_DELTA) * off) <= 1e-12 * off


def test_kappa_estimator_matches_dense(orc):
    """The search's estimator (Hager's method on A^-T with preconditioned
    GMRES solves) against kappa_inf from a dense inverse at n = 1024: a lower
    bound (it is the 1-norm of A^-T times a unit vector) within a factor of
    two here (Higham reports the method within a factor of 3 in practice)."""
    import importlib.util
    import os

    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("condition_random", os.path.join(here, "oracle",
                                                                                   "condition_random.py"))
    cr = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(cr)
    for delta in (0.0, W.RANDOM_DELTA):
        A = W.random_sparse(1024, 16, 2.0, delta=delta)
        est = cr.kappa_inf_estimate(A, W.pattern_power_topk(A, 24))
        D = A.to_scipy().toarray()
        exact = np.abs(D).sum(axis=1).max() * np.abs(np.linalg.inv(D)).sum(axis=1).max()
        assert 0.5 * exact <= est <= exact * (1 + 1e-9), (delta, est, exact)
