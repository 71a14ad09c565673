"""torch.autograd.Function for x = A^-1 b computed by BSPAI-GMRES-IR.

Forward: SPAI build (Alg 2.1, fixed pattern), bucketing (Alg 2.2) and
GMRES-IR (Alg 3.1) for every right-hand side.  Backward, for a loss L(x):
lambda = A^-T dL/dx by BSPAI-GMRES-IR on A^T, left-preconditioned by the
transposed bucketed M; dL/db = lambda and dL/dA_ij = -lambda_i x_j on the
nonzeros of A.  The preconditioner is a function of A but does not change the
solution, so no derivative flows through it.  Every step runs in the CUDA
library through the C ABI; this module only sequences the calls.
"""
from __future__ import annotations

import queue
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import torch

from . import bspai as B


@dataclass
class SolverSettings:
    spai_eps: float = 0.3
    bucket_eps: float = 2.0 ** -16
    precs: list = field(default_factory=lambda: ["fp64", "fp32", "fp16"])
    u_g: str = "fp32"
    u_p: str = "fp32"
    tol: float = 1e-4
    # right-hand sides solved at the same time, each on its own CUDA stream with
    # its cooperative GMRES kernels capped at (SM count / concurrent) blocks
    concurrent: int = 16
    # device bytes the Krylov basis of one solve may take (bspai_opts_t
    # basis_bytes_max); None: half of the device's free memory shared among the
    # concurrent solves.  Where kmax + 1 vectors do not fit, each refinement step
    # runs restarted GMRES cycles that rebuild a smaller basis instead of storing
    # the whole one.
    basis_bytes_max: int | None = None


def _basis_cap(settings: SolverSettings, device, k: int) -> int:
    if settings.basis_bytes_max is not None:
        return int(settings.basis_bytes_max)
    free, _ = torch.cuda.mem_get_info(device)
    return max(1, free // (2 * k))


def _solve_rhs(Ah, rhs, BM, M, out, settings: SolverSettings, what: str):
    """out[r] = A^-1 rhs[r] by BSPAI-GMRES-IR for every row r, several at once."""
    nr = rhs.shape[0]
    k = max(1, min(nr, settings.concurrent))
    cap = _basis_cap(settings, rhs.device, k)
    if k == 1:
        o = B.opts(tau=settings.tol, basis_bytes_max=cap)
        infos = [B.gmres_ir_solve(Ah, rhs[r], BM, M, out[r], u_g=settings.u_g, u_p=settings.u_p, tol=settings.tol,
                                  o=o) for r in range(nr)]
    else:
        sms = torch.cuda.get_device_properties(rhs.device).multi_processor_count
        o = B.opts(tau=settings.tol, max_blocks=max(1, sms // k), basis_bytes_max=cap)
        main = torch.cuda.current_stream()
        streams = queue.Queue()
        for _ in range(k):
            st = torch.cuda.Stream()
            st.wait_stream(main)
            streams.put(st)

        def one(r):
            st = streams.get()
            try:
                # the library works on the calling thread's current device
                torch.cuda.set_device(rhs.device)
                return B.gmres_ir_solve(Ah, rhs[r], BM, M, out[r], u_g=settings.u_g, u_p=settings.u_p,
                                        tol=settings.tol, o=o, stream=st)
            finally:
                streams.put(st)

        with ThreadPoolExecutor(k) as ex:
            infos = list(ex.map(one, range(nr)))
        while not streams.empty():
            main.wait_stream(streams.get())
    for r, info in enumerate(infos):
        if info["status"] != B.OK:
            raise B.BspaiError(info["status"], f"{what} solve of right-hand side {r}: {info}")
    return infos


class BspaiSolve(torch.autograd.Function):
    """x = BspaiSolve.apply(a_val, b, row_ptr, col, pattern, settings)

    a_val: (nnz,) float64 CUDA tensor, the values of A in CSR order;
    b: (n,) or (nrhs, n) float64 CUDA tensor; row_ptr, col: int32 CUDA
    tensors of A's CSR structure; pattern: DeviceCSR of M's pattern."""

    @staticmethod
    def forward(ctx, a_val, b, row_ptr, col, pattern, settings: SolverSettings):
        n = int(row_ptr.numel() - 1)
        A = B.DeviceCSR(n, row_ptr, col, a_val.detach().contiguous())
        Ah = B.matrix_create(A)
        M, _ = B.bspai_build(A, pattern, settings.spai_eps)
        BM, _ = B.bspai_bucket(M, settings.bucket_eps, settings.precs)
        bb = b.detach().reshape(-1, n).contiguous()
        x = torch.empty_like(bb)
        infos = _solve_rhs(Ah, bb, BM, M, x, settings, "forward")
        ctx.handles = (A, Ah, M, BM, settings)
        ctx.infos = infos
        ctx.b_shape = b.shape
        ctx.save_for_backward(x)
        return x.reshape(b.shape)

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        A, Ah, M, BM, settings = ctx.handles
        n = A.n
        At = B.matrix_transpose(Ah)
        Mt = B.M_transpose(M)
        BMt = B.bucket_transpose(BM)
        g = gx.detach().reshape(-1, n).contiguous()
        lam = torch.empty_like(g)
        grad_a = torch.empty_like(A.val)
        ctx.adjoint_infos = _solve_rhs(At, g, BMt, Mt, lam, settings, "adjoint")
        B.adjoint_grad_A(A, lam, x, grad_a)
        return grad_a, lam.reshape(ctx.b_shape), None, None, None, None


def solve(a_val, b, row_ptr, col, pattern, settings: SolverSettings | None = None):
    """Differentiable x = A^-1 b (see BspaiSolve)."""
    return BspaiSolve.apply(a_val, b, row_ptr, col, pattern, settings or SolverSettings())
