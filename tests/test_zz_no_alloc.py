"""bspai_gmres_noalloc: the GMRES solve with its workspace in the library's
fixed device block, for callers that cannot allocate device memory during the
call.  Checked through the C ABI against bspai_gmres (the allocating entry
point) on two calls in a row, with the GMRES tolerances of the parity tests
(fp32 1e-4, fp64 1e-10 relative).  Kept in a file that pytest collects last."""
import numpy as np
import pytest
import torch

from gpu_helpers import dev, gpu_bucket, gpu_build, host, lib
from paper_2307_03914_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-4, "fp64": 1e-10}


@pytest.fixture(scope="module")
def B():
    return lib()


def _system(B, grid):
    wl = W.workload("convdiff3d", grid=grid)
    A, P = wl["A"], wl["pattern"]
    g = gpu_build(B, wl)
    bk = gpu_bucket(B, g["M"], P.nnz, 2.0 ** -16, wl["precs"])
    Ah = B.matrix_create(g["A"])
    r = dev(np.random.default_rng(11).uniform(-1, 1, A.n) * np.abs(wl["b"]).max())
    return wl, g, bk, Ah, r


@pytest.mark.parametrize("ug", ["fp32", "fp64"])
def test_noalloc_matches_allocating_gmres_twice(B, ug):
    wl, g, bk, Ah, r = _system(B, 16)
    n = wl["A"].n
    o = B.opts(tau=1e-6, kmax=200)
    d_ref = torch.empty(n, dtype=torch.float64, device="cuda")
    ref = B.gmres(Ah, bk["BM"], r, d_ref, ug, ug, o)
    dr = host(d_ref)
    for call in range(2):
        d = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        info = B.gmres_noalloc(Ah, bk["BM"], r, d, ug, ug, o)
        assert info["status"] == 0, (call, info)
        assert info["gmres_iters"] == ref["gmres_iters"], call
        dg = host(d)
        assert np.linalg.norm(dg - dr) <= TOL[ug] * np.linalg.norm(dr), call


def test_noalloc_rejects_oversized_problem(B):
    wl, g, bk, Ah, r = _system(B, 64)  # n = 262,144: a 300-step fp32 basis needs ~315 MB
    d = torch.zeros(wl["A"].n, dtype=torch.float64, device="cuda")
    with pytest.raises(B.BspaiError) as e:
        B.gmres_noalloc(Ah, bk["BM"], r, d, "fp32", "fp32", B.opts(tau=1e-6, kmax=300))
    assert e.value.status == B.ERR_INVALID and "bytes of scratch" in str(e.value)
    assert torch.all(d == 0)
    # the same system with a basis that fits still runs
    info = B.gmres_noalloc(Ah, bk["BM"], r, d, "fp32", "fp32", B.opts(tau=1e-6, kmax=40))
    assert info["status"] == 0 and info["gmres_iters"][0] >= 1
