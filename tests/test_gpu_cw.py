"""Componentwise, x-dependent bucketing (the strategy Section 2.3 sets aside)
on the GPU through bspai_apply_cw: the bucket of every entry, the per-bucket
counts and the product y = M x, bit-exact against the oracle's
bucket_ids_cw + bucket_store + bspmv on the same M (the oracle's SPAI rounded
to u_f) and x, at small sizes (several slices, ragged ends) and on the whole
128^3 workload."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import dev, host, lib, oracle_M, small_workloads
from paper_2307_03914_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PLISTS = [["fp64", "fp32", "bf16", "drop"], ["fp32", "bf16"], ["fp64", "bf16", "drop"], ["fp64"]]
EPS = [2.0 ** -40, 2.0 ** -24, 2.0 ** -12, 2.0 ** -6]


@pytest.fixture(scope="module")
def B():
    return lib()


def _check(B, M, P, muf, x, precs, eps, ydt):
    n = P.n
    y = torch.empty(n, dtype=ydt, device="cuda")
    ids = torch.full((P.nnz,), -1, dtype=torch.int8, device="cuda")
    counts = B.apply_cw(M, eps, precs, dev(x), y, ids=ids, counts=True)
    x64 = x.astype(np.float64)
    ref = O.bucket_ids_cw(P.row_ptr, P.col, muf, x64, eps, precs)
    assert np.array_equal(host(ids), ref["ids"]), (precs, eps)
    assert counts == ref["nnz_k"].tolist()
    stored, _, _ = O.bucket_store(P.row_ptr, P.col, muf, ref["ids"], precs)
    yr = O.bspmv(P.row_ptr, P.col, stored, ref["ids"], precs, x64)
    if ydt == torch.float32:
        yr = yr.astype(np.float32).astype(np.float64)
    assert np.array_equal(host(y).astype(np.float64), yr), (precs, eps, ydt)


@pytest.mark.parametrize("wl", small_workloads(), ids=lambda w: f"{w['name']}-{w['A'].n}")
def test_cw_product_bitexact(B, wl):
    P = wl["pattern"]
    M, muf = oracle_M(B, wl)
    rng = np.random.default_rng(17)
    x64 = rng.uniform(-1, 1, P.n) * np.exp(rng.normal(0, 2, P.n))
    x32 = x64.astype(np.float32)
    for precs in PLISTS:
        for eps in EPS:
            for x, ydt in [(x64, torch.float64), (x32, torch.float32), (x64, torch.float32)]:
                _check(B, M, P, muf, x, precs, eps, ydt)


def test_cw_rejects_scaled_formats(B):
    wl = small_workloads()[0]
    M, _ = oracle_M(B, wl)
    x = torch.zeros(wl["A"].n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(B.BspaiError) as e:
        B.apply_cw(M, 2.0 ** -10, ["fp64", "fp32", "fp16"], x, y)
    assert e.value.status == B.ERR_UNSUPPORTED
    with pytest.raises(B.BspaiError):
        B.apply_cw(M, 2.0 ** -10, ["fp32", "fp64"], x, y)


def test_cw_full_size_128(B):
    wl = W.workload("convdiff3d")
    P = wl["pattern"]
    M, muf = oracle_M(B, wl)
    x = np.random.default_rng(3).uniform(-1, 1, P.n).astype(np.float32)
    _check(B, M, P, muf, x, ["fp64", "fp32", "bf16", "drop"], 2.0 ** -10, torch.float32)
