"""The kernel forms of the sparse products -- compile-time bucket formats
(default), the generic register form, and the form that stages the matrix
stream into shared memory with bulk copies (TMA) -- on matrices large enough
for the staged form to engage (more than 2 x 8 x 152 slices of 32 rows): each
bit-exact against the oracle's Alg 2.3 product and its u_p product, for every
bucket mix (1 to 4 stored buckets, an fp64 bucket or none, rows wider than the
unrolled part, a ragged last slice), and GMRES iterates identical between the
forms."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import dev, gpu_bucket, host, lib, oracle_M
from paper_2307_03914_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FORMS = (0, 1, 2)  # SPMV_AUTO, SPMV_REGISTERS, SPMV_STAGED


@pytest.fixture(scope="module")
def B():
    b = lib()
    yield b
    b.set_spmv_form(b.SPMV_AUTO)


def _wl3d(dims):
    A = W.convdiff3d(dims, (1.0, 10.0, 100.0), 0.8)
    x, b = W.rhs(A)
    return dict(name=f"convdiff3d_{dims}", A=A, pattern=W.pattern_of(A), x_true=x, b=b, spai_eps=0.3,
                precs=["fp64", "fp32", "fp16", "e4m3"], tau=1e-4, u_g="fp32", u_p="fp32")


@pytest.fixture(scope="module")
def cases(B):
    out = []
    for wl in [_wl3d((47, 48, 49)), W.workload("random", n=90000)]:
        M, muf = oracle_M(B, wl)
        out.append((wl, M, muf))
    return out


MIXES = [
    (["fp64", "fp32", "fp16", "e4m3"], 2.0 ** -10),   # fp16 + e4m3 stored (the bench mix)
    (["fp64", "fp32", "fp16"], 2.0 ** -28),            # fp64 + fp32 + fp16 stored
    (["fp64", "fp32", "fp16", "bf16"], 2.0 ** -30),    # up to four stored, fp64 first
    (["fp32", "fp16"], 2.0 ** -12),                    # no fp64 bucket
    (["fp64"], 2.0 ** -53),                            # q = 1: one fp64 bucket
]


def _apply(B, BM, xin, ydt, form):
    B.set_spmv_form(form)
    y = torch.empty(xin.shape[0], dtype=ydt, device="cuda")
    B.apply(BM, dev(xin), y)
    return host(y).astype(np.float64)


@pytest.mark.parametrize("mix", range(len(MIXES)))
def test_bucketed_product_forms_bitexact(B, cases, mix):
    precs, eps = MIXES[mix]
    for wl, M, muf in cases:
        P = wl["pattern"]
        b = gpu_bucket(B, M, P.nnz, eps, precs)
        ref = O.bucket_ids(P.row_ptr, muf, eps, precs)
        stored, _, _ = O.bucket_store(P.row_ptr, P.col, muf, ref["ids"], precs)
        rng = np.random.default_rng(11)
        x64 = rng.uniform(-1, 1, P.n)
        x32 = rng.uniform(-1, 1, P.n).astype(np.float32)
        for xin, ydt in [(x32, torch.float32), (x64, torch.float32), (x64, torch.float64)]:
            yr = O.bspmv(P.row_ptr, P.col, stored, ref["ids"], precs, xin.astype(np.float64))
            if ydt == torch.float32:
                yr = yr.astype(np.float32).astype(np.float64)
            for form in FORMS:
                yg = _apply(B, b["BM"], xin, ydt, form)
                assert np.array_equal(yg, yr), (wl["name"], precs, eps, ydt, form)


def test_up_product_and_x0_forms_bitexact(B, cases):
    for wl, M, muf in cases:
        A, P = wl["A"], wl["pattern"]
        Ah = B.matrix_create(B.DeviceCSR.from_host(A))
        v = np.random.default_rng(12).uniform(-1, 1, A.n).astype(np.float32)
        ref = O.spmv_prec(A.row_ptr, A.col, A.val, "fp32", v.astype(np.float64))
        x0r = O.spmv_prec(P.row_ptr, P.col, muf, "fp32", wl["b"])
        for form in FORMS:
            B.set_spmv_form(form)
            w = torch.empty(A.n, dtype=torch.float32, device="cuda")
            B.spmv_up(Ah, dev(v), w)
            assert np.array_equal(host(w).astype(np.float64), ref), (wl["name"], form)
            y = torch.empty(P.n, dtype=torch.float64, device="cuda")
            B.apply_uf(M, dev(wl["b"]), y)
            assert np.array_equal(host(y), x0r), (wl["name"], form)


def test_gmres_iterates_identical_between_forms(B, cases):
    wl, M, muf = cases[0]
    A, P = wl["A"], wl["pattern"]
    b = gpu_bucket(B, M, P.nnz, 2.0 ** -10, wl["precs"])
    Ah = B.matrix_create(B.DeviceCSR.from_host(A))
    r = dev(O.residual_dd(A, O.spmv_prec(P.row_ptr, P.col, muf, "fp32", wl["b"]), wl["b"]))
    out = []
    for form in FORMS:
        B.set_spmv_form(form)
        d = torch.empty(A.n, dtype=torch.float64, device="cuda")
        info = B.gmres(Ah, b["BM"], r, d, "fp32", "fp32", B.opts(tau=1e-4))
        out.append((host(d), info["gmres_iters"]))
    B.set_spmv_form(B.SPMV_AUTO)
    for d, its in out[1:]:
        assert its == out[0][1]
        assert np.array_equal(d, out[0][0])
