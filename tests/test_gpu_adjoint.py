"""GPU adjoint (differentiation extension): transposed operators bit-exact
against the oracle on the transposed inputs, lambda = A^-T g against the
oracle's fp64 adjoint (1e-10), and the autograd gradients dL/db, dL/dA
against central finite differences of the GPU forward solve (1e-5)."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import dev, gpu_bucket, host, lib, oracle_M
from paper_2307_03914_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [("diffusion2d", 32), ("convdiff2d", 21), ("convdiff3d", 9)]


@pytest.fixture(scope="module")
def B():
    return lib()


@pytest.mark.parametrize("name,grid", CASES)
def test_transposed_operators_bitexact(B, name, grid):
    wl = W.workload(name, grid=grid)
    A, P = wl["A"], wl["pattern"]
    n = A.n
    trp, tcol, tval = O.transpose_csr(A.row_ptr, A.col, A.val)
    Ah = B.matrix_create(B.DeviceCSR.from_host(A))
    At = B.matrix_transpose(Ah)
    rng = np.random.default_rng(5)
    v = rng.uniform(-1, 1, n).astype(np.float32)
    w = torch.empty(n, dtype=torch.float32, device="cuda")
    B.spmv_up(At, dev(v), w)
    assert np.array_equal(host(w).astype(np.float64), O.spmv_prec(trp, tcol, tval, "fp32", v.astype(np.float64)))
    x = rng.uniform(-1, 1, n)
    r = torch.empty(n, dtype=torch.float64, device="cuda")
    B.residual(At, dev(x), dev(wl["b"]), r)
    assert np.array_equal(host(r), O.residual_dd(W.CSR(n, trp, tcol, tval), x, wl["b"]))
    # M^T in u_f and the transposed bucketed M, from the oracle's M
    M, muf = oracle_M(B, wl)
    mrp, mcol, mval = O.transpose_csr(P.row_ptr, P.col, muf)
    Mt = B.M_transpose(M)
    rp_, col_, val_, _ = B.M_export(Mt, n, P.nnz)
    assert np.array_equal(host(rp_), mrp) and np.array_equal(host(col_), mcol)
    assert np.array_equal(host(val_).astype(np.float64), mval)
    for precs, eps in [(wl["precs"], 2.0 ** -16), (["fp64", "fp32", "fp16", "e4m3", "drop"], 2.0 ** -12),
                       (["fp32", "bf16", "e4m3"], 2.0 ** -10)]:
        bk = gpu_bucket(B, M, P.nnz, eps, precs)
        ids = O.bucket_ids(P.row_ptr, muf, eps, precs)["ids"]
        stored, _, _ = O.bucket_store(P.row_ptr, P.col, muf, ids, precs)
        # transpose the stored values and the ids with the same permutation
        _, _, perm = O.transpose_csr(P.row_ptr, P.col, np.arange(P.nnz, dtype=np.float64))
        perm = perm.astype(np.int64)
        BMt = B.bucket_transpose(bk["BM"])
        for xin, ydt in [(rng.uniform(-1, 1, n), torch.float64), (rng.uniform(-1, 1, n).astype(np.float32),
                                                                   torch.float32)]:
            y = torch.empty(n, dtype=ydt, device="cuda")
            B.apply(BMt, dev(xin), y)
            yr = O.bspmv(mrp, mcol, stored[perm], ids[perm], precs, xin.astype(np.float64))
            if ydt == torch.float32:
                yr = yr.astype(np.float32).astype(np.float64)
            assert np.array_equal(host(y).astype(np.float64), yr), (precs, eps, ydt)


def _problem(B, name, grid, nrhs=1, seed=0):
    wl = W.workload(name, grid=grid)
    A, P = wl["A"], wl["pattern"]
    rng = np.random.default_rng(seed)
    xs = rng.uniform(-1, 1, (nrhs, A.n))
    bs = (A.to_scipy() @ xs.T).T
    xt = rng.uniform(-1, 1, (nrhs, A.n))
    rp, col = dev(A.row_ptr.astype(np.int32)), dev(A.col.astype(np.int32))
    Pd = B.DeviceCSR.from_host(P, with_values=False)
    return wl, A, P, bs, xt, rp, col, Pd


@pytest.mark.parametrize("name,grid", CASES[:2])
def test_adjoint_matches_oracle_and_finite_differences(B, name, grid):
    from paper_2307_03914_gb300 import autograd as AG

    wl, A, P, bs, xt, rp, col, Pd = _problem(B, name, grid)
    st = AG.SolverSettings(spai_eps=wl["spai_eps"], bucket_eps=2.0 ** -16, precs=wl["precs"])
    aval = dev(A.val).requires_grad_(True)
    b = dev(bs[0]).requires_grad_(True)
    xtd = dev(xt[0])
    x = AG.solve(aval, b, rp, col, Pd, st)
    loss = ((x - xtd) ** 2).sum()
    loss.backward()
    gb, gA = host(b.grad), host(aval.grad)
    # the oracle's fp64 adjoint on its own forward solution
    muf = O.round_to(O.spai(A, P, wl["spai_eps"])["mval"], "fp32")
    S = O.System(A, P.row_ptr, P.col, muf, np.zeros(P.nnz, np.int8), ["fp64"])
    xo = O.gmres_ir(S, muf, bs[0], "fp64", "fp64", 1e-12, 500, 10)["x"]
    adj = O.adjoint(A, P, muf, xo, 2 * (xo - xt[0]))
    assert np.abs(gb - adj["db"]).max() <= 1e-10 * np.abs(adj["db"]).max()
    assert np.abs(gA - adj["dA"]).max() <= 1e-10 * np.abs(adj["dA"]).max()

    # central finite differences of the GPU forward solve
    def L(av, bv):
        with torch.no_grad():
            xx = AG.solve(av, bv, rp, col, Pd, st)
            return float(((xx - xtd) ** 2).sum())

    rng = np.random.default_rng(9)
    for i in rng.choice(A.n, 4, replace=False):
        h = 1e-6 * max(1.0, abs(bs[0][i]))
        bp, bm = bs[0].copy(), bs[0].copy()
        bp[i] += h
        bm[i] -= h
        fd = (L(aval.detach(), dev(bp)) - L(aval.detach(), dev(bm))) / (2 * h)
        assert abs(fd - gb[i]) <= 1e-5 * max(abs(fd), 1e-3), (i, fd, gb[i])
    for p in rng.choice(A.nnz, 4, replace=False):
        h = 1e-6 * max(1.0, abs(A.val[p]))
        ap, am = A.val.copy(), A.val.copy()
        ap[p] += h
        am[p] -= h
        fd = (L(dev(ap), b.detach()) - L(dev(am), b.detach())) / (2 * h)
        assert abs(fd - gA[p]) <= 1e-5 * max(abs(fd), 1e-3), (p, fd, gA[p])


def test_adjoint_with_a_capped_krylov_basis(B):
    """Krylov bases recomputed instead of stored: with the basis capped at 12
    vectors, the forward and adjoint solves restart their GMRES cycles, and the
    gradients still match the oracle's adjoint (solved with the same cap) and the
    uncapped GPU gradients to 1e-10."""
    from paper_2307_03914_gb300 import autograd as AG

    wl, A, P, bs, xt, rp, col, Pd = _problem(B, "convdiff2d", 21, nrhs=2, seed=4)
    kmem = 11
    cap = (kmem + 1) * 4 * (-(-A.n // 64) * 64)  # u_g = fp32 vectors, rows rounded up to 64

    def grads(basis):
        st = AG.SolverSettings(spai_eps=wl["spai_eps"], bucket_eps=2.0 ** -16, precs=wl["precs"],
                               basis_bytes_max=basis)
        aval = dev(A.val).requires_grad_(True)
        b = dev(bs).requires_grad_(True)
        x = AG.solve(aval, b, rp, col, Pd, st)
        loss = ((x - dev(xt)) ** 2).sum()
        loss.backward()
        return host(b.grad), host(aval.grad), x.grad_fn

    gb, gA, fn = grads(cap)
    assert all(i["kmem"] == kmem for i in fn.adjoint_infos + fn.infos)
    assert max(max(i["gmres_cycles"]) for i in fn.adjoint_infos) > 1
    gb0, gA0, _ = grads(None)
    assert np.abs(gb - gb0).max() <= 1e-10 * np.abs(gb0).max()
    assert np.abs(gA - gA0).max() <= 1e-10 * np.abs(gA0).max()
    muf = O.round_to(O.spai(A, P, wl["spai_eps"])["mval"], "fp32")
    S = O.System(A, P.row_ptr, P.col, muf, np.zeros(P.nnz, np.int8), ["fp64"])
    for r in range(2):
        xo = O.gmres_ir(S, muf, bs[r], "fp64", "fp64", 1e-12, 500, 10)["x"]
        adj = O.adjoint(A, P, muf, xo, 2 * (xo - xt[r]), kmem=kmem)
        assert max(adj["info"]["cycles"]) > 1
        assert np.abs(gb[r] - adj["db"]).max() <= 1e-10 * np.abs(adj["db"]).max()


def test_adjoint_full_size_16_rhs(B):
    """2D diffusion 256^2 with a log-normal coefficient field, 16 right-hand
    sides: every adjoint solution satisfies A^T lambda = g to the level of u,
    and sampled gradients match central finite differences."""
    from paper_2307_03914_gb300 import autograd as AG

    wl, A, P, bs, xt, rp, col, Pd = _problem(B, "diffusion2d", 256, nrhs=16, seed=1)
    st = AG.SolverSettings(spai_eps=wl["spai_eps"], bucket_eps=2.0 ** -16, precs=wl["precs"])
    aval = dev(A.val).requires_grad_(True)
    b = dev(bs).requires_grad_(True)
    xtd = dev(xt)
    x = AG.solve(aval, b, rp, col, Pd, st)
    loss = ((x - xtd) ** 2).sum()
    loss.backward()
    lam = b.grad.detach()
    g = 2 * (x.detach() - xtd)
    Ah = B.matrix_create(B.DeviceCSR.from_host(A))
    At = B.matrix_transpose(Ah)
    r = torch.empty(A.n, dtype=torch.float64, device="cuda")
    anorm = np.abs(A.to_scipy()).sum(axis=0).max()  # ||A^T||_inf
    for k in range(16):
        B.residual(At, lam[k], g[k], r)
        nbe = float(r.abs().max()) / (anorm * float(lam[k].abs().max()) + float(g[k].abs().max()))
        assert nbe <= 4 * 2.0 ** -53, (k, nbe)
    gb = host(b.grad)
    gA = host(aval.grad)

    def L(av, bv):
        with torch.no_grad():
            xx = AG.solve(av, bv, rp, col, Pd, st)
            return float(((xx - xtd) ** 2).sum())

    i = 12345
    h = 1e-6 * max(1.0, abs(bs[3][i]))
    bp, bm = bs.copy(), bs.copy()
    bp[3, i] += h
    bm[3, i] -= h
    fd = (L(aval.detach(), dev(bp)) - L(aval.detach(), dev(bm))) / (2 * h)
    assert abs(fd - gb[3, i]) <= 1e-5 * max(abs(fd), 1e-3)
    p = A.row_ptr[30000] + 1
    h = 1e-6 * max(1.0, abs(A.val[p]))
    ap, am = A.val.copy(), A.val.copy()
    ap[p] += h
    am[p] -= h
    fd = (L(dev(ap), b.detach()) - L(dev(am), b.detach())) / (2 * h)
    assert abs(fd - gA[p]) <= 1e-5 * max(abs(fd), 1e-3)


def test_adjoint_grad_multi_rhs_bitexact(B):
    """dL/dA summed over right-hand sides inside the kernel, bit-exact against
    the oracle's sum (r ascending, one rounding per product and per sum)."""
    wl = W.workload("diffusion2d", grid=32)
    A = wl["A"]
    rng = np.random.default_rng(21)
    Ad = B.DeviceCSR.from_host(A)
    for nrhs in (1, 3, 16):
        lam = rng.uniform(-1, 1, (nrhs, A.n))
        x = rng.uniform(-1, 1, (nrhs, A.n))
        dA = torch.full((A.nnz,), np.nan, dtype=torch.float64, device="cuda")
        B.adjoint_grad_A(Ad, dev(lam if nrhs > 1 else lam[0]), dev(x if nrhs > 1 else x[0]), dA)
        assert np.array_equal(host(dA), O.adjoint_grad_A(A, lam, x)), nrhs
