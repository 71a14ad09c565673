"""Pins for the oracle's memory-capped inner solve: when the Krylov basis may
hold only kmem + 1 vectors, each refinement step (Alg 3.1) solves its
correction equation by restarted GMRES cycles.  Checked against what the
mathematics fixes: the refinement's fixed point (a dense solve), the
minimal-residual property of every cycle, the exact-inverse special case and
the step bounds; and against the uncapped driver when the cap does not bind."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2307_03914_gb300 import workloads as W


def _csr(Ad):
    S = sp.csr_matrix(Ad)
    S.sort_indices()
    return W.CSR(Ad.shape[0], S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(float))


def _system(orc, A, Mdense):
    Mc = _csr(Mdense)
    return orc.System(A, Mc.row_ptr, Mc.col, Mc.val, np.zeros(Mc.nnz, np.int8), ["fp64"])


def _spai_system(orc, A, P, eps=0.3):
    muf = orc.round_to(orc.spai(A, P, eps)["mval"], "fp32")
    bk = orc.bucket_ids(P.row_ptr, muf, 2.0 ** -53, ["fp64"])
    st, _, _ = orc.bucket_store(P.row_ptr, P.col, muf, bk["ids"], ["fp64"])
    return orc.System(A, P.row_ptr, P.col, st, bk["ids"], ["fp64"]), muf


def test_cap_that_does_not_bind_changes_nothing(orc):
    wl = W.workload("convdiff2d")
    ref = orc.solve(wl)
    cap = orc.solve(wl, kmem=max(ref["its"]))
    assert np.array_equal(cap["x"], ref["x"]) and cap["its"] == ref["its"]
    assert cap["cycles"] == [1] * len(ref["its"])


@pytest.mark.parametrize("kmem", [2, 5, 12])
def test_capped_refinement_reaches_the_dense_solution(orc, kmem):
    """Whatever the inner solver, refinement in u = fp64 with a Dot2 residual
    converges to x = A^-1 b to the level of u: the capped driver's x agrees with
    a dense LU solve and with the uncapped driver."""
    A = W.convdiff2d(12, 12, (0.6, 0.3))
    P = W.pattern_of(A)
    S, muf = _spai_system(orc, A, P)
    Ad = A.to_scipy().toarray()
    xt = np.random.default_rng(kmem).uniform(-1, 1, A.n)
    b = Ad @ xt
    ref = np.linalg.solve(Ad, b)
    out = orc.gmres_ir(S, muf, b, "fp64", "fp64", 1e-6, kmax=300, imax=30, kmem=kmem)
    full = orc.gmres_ir(S, muf, b, "fp64", "fp64", 1e-6, kmax=300, imax=30)
    kappa = np.linalg.cond(Ad, np.inf)
    assert np.abs(out["x"] - ref).max() <= 4 * kappa * 2.0 ** -53 * np.abs(ref).max()
    assert np.abs(out["x"] - full["x"]).max() <= 4 * kappa * 2.0 ** -53 * np.abs(ref).max()
    # the cap binds: some step restarts, and every step obeys the step bounds
    assert max(out["cycles"]) > 1
    for its, c in zip(out["its"], out["cycles"]):
        assert c <= -(-300 // kmem) and (c - 1) * kmem <= its <= c * kmem


def test_each_cycle_does_not_increase_the_preconditioned_residual(orc):
    """GMRES minimises ||M (r - A d)||_2 over d_prev + K_m: a further cycle never
    raises it (fp64 arithmetic, up to rounding).  x0 = 0 and one refinement step,
    so x is the restarted solve's own correction after c cycles (tau = 0: no
    cycle stops early; kmax = c kmem bounds the cycles)."""
    A = W.convdiff2d(10, 10, (1.0, 0.4))
    P = W.pattern_of(A)
    S, muf = _spai_system(orc, A, P)
    Ad = A.to_scipy().toarray()
    Md = sp.csr_matrix((muf, P.col, P.row_ptr), shape=(A.n, A.n)).toarray()
    b = np.random.default_rng(3).uniform(-1, 1, A.n)
    kmem = 3
    prev = np.linalg.norm(Md @ b)
    for c in range(1, 7):
        out = orc.gmres_ir(S, muf, b, "fp64", "fp64", 0.0, kmax=c * kmem, imax=1, x0=np.zeros(A.n), kmem=kmem)
        assert out["cycles"] == [c] and out["its"] == [c * kmem]
        res = np.linalg.norm(Md @ (b - Ad @ out["x"]))
        assert res <= prev * (1 + 1e-12), (c, res, prev)
        assert res < prev  # and strictly here: the cycles make progress on this system
        prev = res


def test_exact_inverse_needs_one_step_whatever_the_cap(orc):
    A = W.convdiff2d(6)
    Ainv = np.linalg.inv(A.to_scipy().toarray())
    S = _system(orc, A, Ainv)
    b = np.random.default_rng(5).uniform(-1, 1, A.n)
    for kmem in (1, 2, 7):
        out = orc.gmres_ir(S, Ainv, b, "fp64", "fp64", 1e-10, kmax=A.n, imax=3, x0=np.zeros(A.n), kmem=kmem)
        assert out["its"][0] == 1 and out["cycles"][0] == 1
