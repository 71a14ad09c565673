"""Pins for the oracle's adjoint (lambda = A^-T g, dL/db = lambda,
dL/dA_ij = -lambda_i x_j) against dense solves and central finite differences
of the loss L = ||x(A, b) - x_target||^2 computed with the oracle's own solver."""
import numpy as np
import pytest

from paper_2307_03914_gb300 import workloads as W


def _setup(orc, wl):
    sp = orc.spai(wl["A"], wl["pattern"], wl["spai_eps"])
    muf = orc.round_to(sp["mval"], "fp32")
    return muf


def _fwd(orc, wl, muf, aval, b):
    A = W.CSR(wl["A"].n, wl["A"].row_ptr, wl["A"].col, aval)
    P = wl["pattern"]
    S = orc.System(A, P.row_ptr, P.col, muf, np.zeros(P.nnz, np.int8), ["fp64"])
    return orc.gmres_ir(S, muf, b, "fp64", "fp64", 1e-12, 500, 10)["x"]


@pytest.mark.parametrize("name,grid", [("diffusion2d", 8), ("convdiff2d", 7)])
def test_adjoint_vs_dense(orc, name, grid):
    wl = W.workload(name, grid=grid)
    muf = _setup(orc, wl)
    rng = np.random.default_rng(2)
    x = _fwd(orc, wl, muf, wl["A"].val, wl["b"])
    g = rng.uniform(-1, 1, wl["A"].n)
    adj = orc.adjoint(wl["A"], wl["pattern"], muf, x, g)
    Ad = wl["A"].to_scipy().toarray()
    lam = np.linalg.solve(Ad.T, g)
    assert np.abs(adj["lam"] - lam).max() <= 1e-10 * np.abs(lam).max()
    dA_dense = -np.outer(lam, x)
    rows = np.repeat(np.arange(wl["A"].n), np.diff(wl["A"].row_ptr))
    assert np.allclose(adj["dA"], dA_dense[rows, wl["A"].col], rtol=1e-10, atol=1e-14)


def test_adjoint_vs_central_differences(orc):
    wl = W.workload("convdiff2d", grid=6)
    A = wl["A"]
    muf = _setup(orc, wl)
    xt = np.random.default_rng(3).uniform(-1, 1, A.n)

    def loss(aval, b):
        x = _fwd(orc, wl, muf, aval, b)
        return np.sum((x - xt) ** 2)

    x = _fwd(orc, wl, muf, A.val, wl["b"])
    adj = orc.adjoint(A, wl["pattern"], muf, x, 2 * (x - xt))
    rng = np.random.default_rng(4)
    for i in rng.choice(A.n, 6, replace=False):
        h = 1e-6 * max(1.0, abs(wl["b"][i]))
        bp, bm = wl["b"].copy(), wl["b"].copy()
        bp[i] += h
        bm[i] -= h
        fd = (loss(A.val, bp) - loss(A.val, bm)) / (2 * h)
        assert abs(fd - adj["db"][i]) <= 1e-5 * max(abs(fd), 1e-3), (i, fd, adj["db"][i])
    for p in rng.choice(A.nnz, 6, replace=False):
        h = 1e-6 * max(1.0, abs(A.val[p]))
        ap, am = A.val.copy(), A.val.copy()
        ap[p] += h
        am[p] -= h
        fd = (loss(ap, wl["b"]) - loss(am, wl["b"])) / (2 * h)
        assert abs(fd - adj["dA"][p]) <= 1e-5 * max(abs(fd), 1e-3), (p, fd, adj["dA"][p])


def test_transpose_csr_roundtrip(orc):
    A = W.random_sparse(300, 7, seed=8)
    trp, tcol, tval = orc.transpose_csr(A.row_ptr, A.col, A.val)
    rp, c, v = orc.transpose_csr(trp, tcol, tval)
    assert np.array_equal(rp, A.row_ptr) and np.array_equal(c, A.col) and np.array_equal(v, A.val)
    Ad = A.to_scipy().toarray()
    T = W.CSR(A.n, trp, tcol, tval).to_scipy().toarray()
    assert np.array_equal(T, Ad.T)


def test_adjoint_grad_multi_rhs_pins(orc):
    """The multi-right-hand-side gradient: nrhs = 1 is -lambda_i x_j on every
    nonzero (i, j); on integer-valued inputs the fp64 sum is exact and equals
    the integer sum over r of -lambda_r[i] x_r[j]; a wrong index (lambda_j x_i)
    or a dropped right-hand side fails one of these."""
    wl = W.workload("convdiff2d", grid=7)
    A = wl["A"]
    n = A.n
    rng = np.random.default_rng(9)
    lam1, x1 = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    g1 = orc.adjoint_grad_A(A, lam1, x1)
    for i in range(n):
        for p in range(A.row_ptr[i], A.row_ptr[i + 1]):
            assert g1[p] == -lam1[i] * x1[A.col[p]]
    lam = rng.integers(-1000, 1000, (5, n)).astype(np.float64)
    x = rng.integers(-1000, 1000, (5, n)).astype(np.float64)
    g = orc.adjoint_grad_A(A, lam, x)
    for i in range(n):
        for p in range(A.row_ptr[i], A.row_ptr[i + 1]):
            j = int(A.col[p])
            assert g[p] == float(sum(-int(lam[r, i]) * int(x[r, j]) for r in range(5)))
