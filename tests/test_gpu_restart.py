"""GPU parity of the memory-capped inner solve (bspai_opts_t.basis_bytes_max):
when the Krylov basis may hold only kmem + 1 vectors, every refinement step
runs restarted GMRES cycles on its correction equation.  Against the oracle's
capped driver (oracle/gmres_ir(kmem=...)) on the same inputs: solutions within
1e-12 relative, forward error <= 1e-10, the same refinement steps and GMRES
counts and cycles within the bars of the uncapped parity test; a cap that does
not bind changes no bit."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import dev, gpu_bucket, gpu_build, host, lib, small_workloads

pytestmark = pytest.mark.gpu

WLS = small_workloads()[:4]
IDS = [f"{w['name']}-{w['A'].n}" for w in WLS]
EPS = 2.0 ** -16


@pytest.fixture(scope="module")
def B():
    return lib()


def _cap(n, ug, kmem):
    """Bytes of kmem + 1 Krylov vectors (rows rounded up to 64)."""
    return (kmem + 1) * (4 if ug == "fp32" else 8) * (-(-n // 64) * 64)


def _solve(B, wl, g, b, o):
    x = torch.empty(wl["A"].n, dtype=torch.float64, device="cuda")
    info = B.gmres_ir_solve(g["A"], dev(wl["b"]), b["BM"], g["M"], x, tol=wl["tau"], u_g=wl["u_g"], u_p=wl["u_p"],
                            o=o)
    return host(x), info


@pytest.mark.parametrize("kmem", [4, 9])
@pytest.mark.parametrize("wl", WLS, ids=IDS)
def test_capped_solve_matches_oracle(B, wl, kmem):
    A, P = wl["A"], wl["pattern"]
    g = gpu_build(B, wl)
    b = gpu_bucket(B, g["M"], P.nnz, EPS, wl["precs"])
    # kmax 500 on both sides: the cycles of a step stop after kmax steps in all
    xg, info = _solve(B, wl, g, b, B.opts(tau=wl["tau"], kmax=500, basis_bytes_max=_cap(A.n, wl["u_g"], kmem)))
    ref = O.solve(wl, bucket_eps=EPS, kmem=kmem)
    assert info["status"] == 0 and info["kmem"] == kmem, info
    assert max(ref["cycles"]) > 1 and max(info["gmres_cycles"]) > 1  # the cap binds
    xt = wl["x_true"]
    assert np.abs(xg - xt).max() / np.abs(xt).max() <= 1e-10
    assert np.abs(ref["x"] - xt).max() / np.abs(xt).max() <= 1e-10
    assert np.abs(xg - ref["x"]).max() <= 1e-12 * np.abs(ref["x"]).max()
    assert abs(info["ir_steps"] - ref["steps"]) <= 1
    for i, (a, c) in enumerate(zip(info["gmres_iters"], ref["its"])):
        assert abs(a - c) <= (max(2, 0.1 * c) if i == 0 else max(4, 0.2 * c)), (i, a, c)
    for a, c in zip(info["gmres_cycles"], ref["cycles"]):
        assert abs(a - c) <= max(1, 0.2 * c)
        assert a <= -(-500 // kmem)
    for a, c in zip(info["gmres_iters"], info["gmres_cycles"]):
        assert (c - 1) * kmem <= a <= c * kmem


@pytest.mark.parametrize("wl", WLS[:2], ids=IDS[:2])
def test_cap_that_does_not_bind_changes_no_bit(B, wl):
    A, P = wl["A"], wl["pattern"]
    g = gpu_build(B, wl)
    b = gpu_bucket(B, g["M"], P.nnz, EPS, wl["precs"])
    x0, i0 = _solve(B, wl, g, b, B.opts(tau=wl["tau"]))
    kmax = min(A.n, 1000)
    x1, i1 = _solve(B, wl, g, b, B.opts(tau=wl["tau"], basis_bytes_max=_cap(A.n, wl["u_g"], kmax)))
    assert np.array_equal(x0, x1)
    assert i0["gmres_iters"] == i1["gmres_iters"] and i1["kmem"] == kmax
    assert i1["gmres_cycles"] == [1] * i1["ir_steps"]


def test_cap_below_two_vectors_is_rejected(B):
    wl = WLS[0]
    A, P = wl["A"], wl["pattern"]
    g = gpu_build(B, wl)
    b = gpu_bucket(B, g["M"], P.nnz, EPS, wl["precs"])
    with pytest.raises(B.BspaiError) as e:
        _solve(B, wl, g, b, B.opts(tau=wl["tau"], basis_bytes_max=_cap(A.n, wl["u_g"], 1) - 1))
    assert e.value.status == B.ERR_INVALID and "basis_bytes_max" in str(e.value)
