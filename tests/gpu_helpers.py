"""Shared helpers of the GPU parity tests: run each step through the C-ABI
(via the ctypes binding) and hand back host arrays for comparison."""
import numpy as np
import torch

from paper_2307_03914_gb300 import workloads as W


def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2307_03914_gb300 import build

    build.build()
    from paper_2307_03914_gb300 import bspai

    return bspai


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def gpu_build(B, wl):
    A = B.DeviceCSR.from_host(wl["A"])
    P = B.DeviceCSR.from_host(wl["pattern"], with_values=False)
    M, info = B.bspai_build(A, P, wl["spai_eps"])
    n, nnz = wl["A"].n, wl["pattern"].nnz
    rp, ci, v, res = B.M_export(M, n, nnz)
    return dict(A=A, P=P, M=M, info=info, row_ptr=host(rp), col=host(ci), val=host(v).astype(np.float64),
                resid=host(res).astype(np.float64))


def oracle_M(B, wl):
    """The oracle's SPAI of the workload (fp64, rounded to u_f = fp32), and the
    same matrix handed to the GPU library with bspai_M_create, so that steps
    after the SPAI build are compared on one M that came from the oracle."""
    import oracle as O

    P = wl["pattern"]
    sp = O.spai(wl["A"], P, wl["spai_eps"])
    muf = O.round_to(sp["mval"], "fp32")
    Md = B.DeviceCSR(P.n, dev(P.row_ptr.astype(np.int32)), dev(P.col.astype(np.int32)), dev(muf))
    return B.M_create(Md), muf


def spai_tolerance(kappa, resid, u_f=2.0 ** -24):
    """Per-column bound on the relative error of an SPAI row computed in u_f:
    max(1e-5, 10 u_f (2 kappa + kappa^2 ||s|| / sqrt(1 - ||s||^2))) (first-order
    least-squares perturbation bound with ||Abar mbar|| = sqrt(1 - ||s||^2))."""
    s = np.minimum(resid, 0.999)
    return np.maximum(1e-5, 10 * u_f * (2 * kappa + kappa ** 2 * s / np.sqrt(1 - s ** 2)))


def gpu_bucket(B, M, nnz, eps, precs):
    BM, info = B.bspai_bucket(M, eps, precs)
    ids, stored = B.bucket_export(BM, nnz)
    return dict(BM=BM, info=info, ids=host(ids), stored=host(stored))


def small_workloads():
    """Seeded cases that span several 32-row slices and end in a ragged slice."""
    return [
        W.workload("convdiff2d"),                       # n = 1024
        W.workload("convdiff2d", grid=21),              # n = 441 (ragged)
        W.workload("convdiff3d", grid=12),              # n = 1728
        _ragged3d(),                                    # n = 693 (7 x 9 x 11)
        W.workload("random", n=2000),                   # |J| = 24, shadows of ~300 rows
    ]


def _ragged3d():
    wl = W.workload("convdiff3d", grid=8)
    A = W.convdiff3d((7, 9, 11), (1.0, 10.0, 100.0), 0.8)
    x, b = W.rhs(A)
    wl.update(A=A, pattern=W.pattern_of(A), x_true=x, b=b, name="convdiff3d_7x9x11")
    return wl
