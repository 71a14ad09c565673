"""ctypes binding of libbspai.so (C ABI declared in include/bspai.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of the library.  Vectors and matrices are torch CUDA tensors (PyTorch provides
device memory and streams); calls are enqueued on torch's current stream.
There is no CPU fallback: importing this module fails loudly when the
library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

LIB_PATH = _build.LIB

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libbspai.so is not built ({LIB_PATH}); run paper_2307_03914_gb300.build.build()")

_lib = C.CDLL(LIB_PATH)

OK, ERR_INVALID, ERR_CUDA, ERR_NOMEM, NOT_CONVERGED, RANK_DEFICIENT, NONFINITE, TIMEOUT, ERR_UNSUPPORTED = range(9)
STATUS_NAMES = ["OK", "ERR_INVALID", "ERR_CUDA", "ERR_NOMEM", "NOT_CONVERGED", "RANK_DEFICIENT",
                "NONFINITE", "TIMEOUT", "ERR_UNSUPPORTED"]
PREC = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3, "e4m3": 4, "drop": 5, "dd": 6}
PREC_NAME = {v: k for k, v in PREC.items()}
K_CLASSES = ["spai", "bucket", "spmv_A", "bspmv", "mgs", "residual", "update", "other"]


class BspaiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class CsrT(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p)]


class BuildInfo(C.Structure):
    _fields_ = [("n", C.c_int32), ("max_cols", C.c_int32), ("max_rows", C.c_int32),
                ("n_converged", C.c_int32), ("n_rank_deficient", C.c_int32), ("nnz", C.c_int64),
                ("max_resid", C.c_double), ("n_capped", C.c_int32), ("n_second_tier", C.c_int32),
                ("total_solves", C.c_int64)]


class BucketInfo(C.Structure):
    _fields_ = [("q", C.c_int32), ("precs", C.c_int32 * 8), ("nnz_k", C.c_int64 * 8),
                ("slots_k", C.c_int64 * 8), ("thresholds", C.c_double * 8), ("norm_inf", C.c_double),
                ("storage_pct", C.c_double), ("storage_pct_last8", C.c_double), ("bytes", C.c_int64)]


class Opts(C.Structure):
    _fields_ = [("tau", C.c_double), ("kmax", C.c_int32), ("i_max", C.c_int32), ("x0_given", C.c_int32),
                ("max_blocks", C.c_int32), ("u_stop", C.c_double), ("stagnation", C.c_double),
                ("barrier_timeout_s", C.c_double), ("basis_bytes_max", C.c_int64)]


class SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("ir_steps", C.c_int32), ("stop_reason", C.c_int32),
                ("total_iters", C.c_int32), ("gmres_iters", C.c_int32 * 32), ("nbe", C.c_double * 33),
                ("dx", C.c_double * 32), ("relres", C.c_double * 32), ("kmem", C.c_int32),
                ("gmres_cycles", C.c_int32 * 32)]


class BatchInfo(C.Structure):
    _fields_ = [("pairs", C.c_int32), ("converged", C.c_int32), ("nonfinite", C.c_int32),
                ("ir_launches", C.c_int32), ("max_ir_steps", C.c_int32), ("max_iters", C.c_int32),
                ("total_iters", C.c_int64), ("block_threads", C.c_int32), ("grid", C.c_int32), ("kmax", C.c_int32),
                ("mgs_rows", C.c_int32), ("z_shared_rows", C.c_int32), ("m_schedule", C.c_int32),
                ("team_rows", C.c_int32), ("tuned_candidates", C.c_int32), ("tune_ms", C.c_float),
                ("gmres_bytes", C.c_int64)]


class BatchSchedule(C.Structure):
    _fields_ = [("block_threads", C.c_int32), ("mgs_rows", C.c_int32), ("z_shared_rows", C.c_int32),
                ("m_schedule", C.c_int32), ("team_rows", C.c_int32)]


class Profile(C.Structure):
    _fields_ = [("ms", C.c_double * 8), ("launches", C.c_int64 * 8)]


_vp = C.c_void_p
_i = C.c_int
_d = C.c_double


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("bspai_last_error", C.c_char_p, [])
_sig("bspai_version", _i, [])
_sig("bspai_launch_count", C.c_longlong, [])
_sig("bspai_barrier_selftest", _i, [_i, _i, _d, _vp, C.POINTER(C.c_float)])
_sig("bspai_set_spmv_form", _i, [_i])
_sig("bspai_opts_default", None, [C.POINTER(Opts)])
_sig("bspai_free", _i, [_vp])
_sig("bspai_profile_enable", _i, [_i])
_sig("bspai_profile_read", _i, [C.POINTER(Profile), _i])
_sig("bspai_matrix_create", _i, [C.POINTER(CsrT), _vp, C.POINTER(_vp)])
_sig("bspai_residual", _i, [_vp, _vp, _vp, _vp, _vp])
_sig("bspai_residual_prec", _i, [_vp, _vp, _vp, _i, _i, _vp, _vp])
_sig("bspai_spmv_up", _i, [_vp, _vp, _vp, _vp])
_sig("bspai_build", _i, [C.POINTER(CsrT), C.POINTER(CsrT), _d, _i, _vp, C.POINTER(_vp), C.POINTER(BuildInfo)])
_sig("bspai_M_export", _i, [_vp, _vp, _vp, _vp, _vp, _vp])
_sig("bspai_build_adaptive", _i, [C.POINTER(CsrT), _d, C.c_int32, C.c_int32, C.c_int32, _i, _vp, C.POINTER(_vp),
                                  C.POINTER(BuildInfo)])
_sig("bspai_M_adaptive_export", _i, [_vp, _vp, _vp, _vp])
_sig("bspai_M_create", _i, [C.POINTER(CsrT), _i, _vp, C.POINTER(_vp)])
_sig("bspai_apply_uf", _i, [_vp, _vp, _vp, _vp])
_sig("bspai_bucket", _i, [_vp, _d, C.POINTER(C.c_int32), C.c_int32, _vp, C.POINTER(_vp), C.POINTER(BucketInfo)])
_sig("bspai_bucket_export", _i, [_vp, _vp, _vp, _vp])
_sig("bspai_bucket_batched", _i, [_vp, _vp, C.c_int32, _d, C.POINTER(C.c_int32), C.c_int32, _vp, C.POINTER(_vp),
                                  C.POINTER(BucketInfo)])
_sig("bspai_apply", _i, [_vp, _vp, _i, _vp, _i, _vp])
_sig("bspai_gmres", _i, [_vp, _vp, _vp, _i, _i, C.POINTER(Opts), _vp, _vp, C.POINTER(SolveInfo)])
_sig("bspai_matrix_transpose", _i, [_vp, _vp, C.POINTER(_vp)])
_sig("bspai_M_transpose", _i, [_vp, _vp, C.POINTER(_vp)])
_sig("bspai_bucket_transpose", _i, [_vp, _vp, C.POINTER(_vp)])
_sig("bspai_adjoint_grad_A", _i, [C.POINTER(CsrT), C.c_int32, _vp, _vp, _vp, _vp])
_sig("bspai_probe_fma", _i, [_i, C.c_int32, _vp, C.POINTER(C.c_double), C.POINTER(C.c_float)])


_sig("bspai_apply_cw", _i, [_vp, _d, C.POINTER(C.c_int32), C.c_int32, _vp, _i, _vp, _i, _vp,
                           C.POINTER(C.c_int64), _vp])


class GmresPlan(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("per_thread", C.c_int32), ("block_threads", C.c_int32),
                ("blocks", C.c_int32), ("poll_bulk", C.c_int32)]


_sig("bspai_gmres_plan", _i, [C.c_int32, _i, C.c_int32, C.POINTER(GmresPlan)])
_sig("bspai_gmres_noalloc", _i, [_vp, _vp, _vp, _i, _i, C.POINTER(Opts), _vp, _vp, C.POINTER(SolveInfo)])
_sig("gmres_ir_solve", _i, [C.POINTER(CsrT), _vp, _vp, _vp, _i, _i, _i, _i, _d, C.POINTER(Opts), _vp, _vp,
                            C.POINTER(SolveInfo)])
_sig("gmres_ir_solve_batched", _i, [_vp, _vp, C.c_int32, C.c_int32, _vp, _vp, _vp, _i, _i, _d, C.POINTER(Opts),
                                    _vp, _vp, C.POINTER(BatchInfo), _vp, _vp])
_sig("bspai_batch_schedule_force", _i, [C.POINTER(BatchSchedule)])
_sig("bspai_batch_tune_table", _i, [C.POINTER(BatchSchedule), C.POINTER(C.c_float), C.c_int32,
                                    C.POINTER(C.c_int32)])
_sig("gmres_ir_solve_h", _i, [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _d, C.POINTER(Opts), _vp, _vp,
                              C.POINTER(SolveInfo)])
_sig("bspai_bucket_A", _i, [_vp, _d, C.POINTER(C.c_int32), C.c_int32, _vp, C.POINTER(_vp), C.POINTER(BucketInfo)])
_sig("bspai_gmres_b", _i, [_vp, _vp, _vp, _vp, _i, C.POINTER(Opts), _vp, _vp, C.POINTER(SolveInfo)])
_sig("gmres_ir_solve_hb", _i, [_vp, _vp, _vp, _vp, _vp, _i, _i, _i, _d, C.POINTER(Opts), _vp, _vp,
                               C.POINTER(SolveInfo)])


def last_error() -> str:
    return _lib.bspai_last_error().decode()


def _check(st: int, allow=(OK,)) -> int:
    if st not in allow:
        raise BspaiError(st, last_error())
    return st


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def version() -> int:
    return _lib.bspai_version()


def barrier_selftest(blocks: int, hold: bool, timeout_s: float, stream=None):
    """Runs the bounded grid barrier once; hold=True makes it never release so
    every wait must run out.  Returns (status, kernel milliseconds)."""
    ms = C.c_float(0.0)
    st = _lib.bspai_barrier_selftest(int(blocks), int(bool(hold)), float(timeout_s), _stream(stream), C.byref(ms))
    _check(st, (OK, TIMEOUT))
    return st, float(ms.value)


SPMV_AUTO, SPMV_REGISTERS, SPMV_STAGED = 0, 1, 2


def set_spmv_form(form: int):
    """SPMV_AUTO: compile-time-format kernels for the common bucket mixes;
    SPMV_REGISTERS: always the generic register form; SPMV_STAGED: the
    shared-memory (TMA) staged form where it applies.  Same bits in every form."""
    _check(_lib.bspai_set_spmv_form(int(form)))


def launch_count() -> int:
    """Kernel launches issued by the library since it was loaded."""
    return int(_lib.bspai_launch_count())


# --------------------------------------------------------------- containers
class DeviceCSR:
    """CSR in device memory: row_ptr/col int32, val float64 (or None)."""

    def __init__(self, n, row_ptr, col, val=None):
        self.n = int(n)
        self.row_ptr, self.col, self.val = row_ptr, col, val

    @classmethod
    def from_host(cls, A, device="cuda", with_values=True):
        rp = torch.as_tensor(np.ascontiguousarray(A.row_ptr, np.int32)).to(device)
        ci = torch.as_tensor(np.ascontiguousarray(A.col, np.int32)).to(device)
        v = None
        if with_values and A.val is not None:
            v = torch.as_tensor(np.ascontiguousarray(A.val, np.float64)).to(device)
        return cls(A.n, rp, ci, v)

    @property
    def nnz(self):
        return int(self.col.numel())

    def c(self) -> CsrT:
        return CsrT(self.n, self.nnz, self.row_ptr.data_ptr(), self.col.data_ptr(),
                    self.val.data_ptr() if self.val is not None else None)


class _Handle:
    def __init__(self, ptr, keep=None):
        self.ptr = ptr
        self._keep = keep

    def free(self):
        if self.ptr:
            _check(_lib.bspai_free(self.ptr))
            self.ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class AHandle(_Handle):
    pass


class MHandle(_Handle):
    pass


class BMHandle(_Handle):
    pass


def opts(tau=1e-4, kmax=0, i_max=0, x0_given=False, u_stop=0.0, stagnation=0.0, barrier_timeout_s=0.0,
         max_blocks=0, basis_bytes_max=0) -> Opts:
    return Opts(tau, kmax, i_max, int(x0_given), int(max_blocks), u_stop, stagnation, barrier_timeout_s,
                int(basis_bytes_max))


def profile_enable(on: bool = True):
    _check(_lib.bspai_profile_enable(int(on)))


def profile_read(reset: bool = True) -> dict:
    p = Profile()
    _check(_lib.bspai_profile_read(C.byref(p), int(reset)))
    return {K_CLASSES[i]: (p.ms[i], p.launches[i]) for i in range(8)}


# ------------------------------------------------------------------ A
def matrix_create(A: DeviceCSR, stream=None) -> AHandle:
    h = C.c_void_p()
    _check(_lib.bspai_matrix_create(C.byref(A.c()), _stream(stream), C.byref(h)))
    return AHandle(h.value)


def residual(Ah: AHandle, x, b, r, stream=None):
    _check(_lib.bspai_residual(Ah.ptr, _ptr(x), _ptr(b), _ptr(r), _stream(stream)))
    return r


def residual_prec(Ah: AHandle, x, b, r, u_r="dd", u="fp64", stream=None):
    """r = b - A x computed in u_r ("dd" or "fp64") and stored in u ("fp64" or "fp32")."""
    _check(_lib.bspai_residual_prec(Ah.ptr, _ptr(x), _ptr(b), PREC[u_r], PREC[u], _ptr(r), _stream(stream)))
    return r


def spmv_up(Ah: AHandle, v, w, stream=None):
    _check(_lib.bspai_spmv_up(Ah.ptr, _ptr(v), _ptr(w), _stream(stream)))
    return w


# ------------------------------------------------------------------ SPAI
def bspai_build(A: DeviceCSR, P: DeviceCSR, spai_eps: float, u_f: str = "fp32", stream=None):
    h = C.c_void_p()
    info = BuildInfo()
    st = _lib.bspai_build(C.byref(A.c()), C.byref(P.c()), float(spai_eps), PREC[u_f], _stream(stream),
                          C.byref(h), C.byref(info))
    _check(st, (OK, RANK_DEFICIENT))
    d = {f: getattr(info, f) for f, _ in BuildInfo._fields_}
    d["status"] = st
    return MHandle(h.value), d


def bspai_build_adaptive(A: DeviceCSR, spai_eps: float, alpha: int, beta: int = 8, imax_rows: int = 256,
                         u_f: str = "fp32", stream=None):
    """Adaptive SPAI (Alg 2.1, alpha > 0) from the identity pattern."""
    h = C.c_void_p()
    info = BuildInfo()
    st = _lib.bspai_build_adaptive(C.byref(A.c()), float(spai_eps), int(alpha), int(beta), int(imax_rows), PREC[u_f],
                                   _stream(stream), C.byref(h), C.byref(info))
    _check(st, (OK, RANK_DEFICIENT))
    d = {f: getattr(info, f) for f, _ in BuildInfo._fields_}
    d["status"] = st
    return MHandle(h.value), d


def M_adaptive_export(M: MHandle, n: int, nnz: int, stream=None):
    """(step_added int8[nnz], col_info int32[n]) of an adaptively built M."""
    step = torch.empty(max(nnz, 1), dtype=torch.int8, device="cuda")
    cinfo = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    _check(_lib.bspai_M_adaptive_export(M.ptr, _ptr(step), _ptr(cinfo), _stream(stream)))
    return step[:nnz], cinfo[:n]


def M_create(Mcsr: DeviceCSR, u_f: str = "fp32", stream=None) -> MHandle:
    """M handle from given values (CSR, fp64, rounded to u_f)."""
    h = C.c_void_p()
    _check(_lib.bspai_M_create(C.byref(Mcsr.c()), PREC[u_f], _stream(stream), C.byref(h)))
    return MHandle(h.value)


def M_export(M: MHandle, n: int, nnz: int, stream=None):
    dev = "cuda"
    rp = torch.empty(n + 1, dtype=torch.int32, device=dev)
    ci = torch.empty(nnz, dtype=torch.int32, device=dev)
    v = torch.empty(nnz, dtype=torch.float32, device=dev)
    res = torch.empty(n, dtype=torch.float32, device=dev)
    _check(_lib.bspai_M_export(M.ptr, _ptr(rp), _ptr(ci), _ptr(v), _ptr(res), _stream(stream)))
    return rp, ci, v, res


def apply_uf(M: MHandle, x, y, stream=None):
    _check(_lib.bspai_apply_uf(M.ptr, _ptr(x), _ptr(y), _stream(stream)))
    return y


# ------------------------------------------------------------------ buckets
def bspai_bucket(M: MHandle, bucket_eps: float, precs, stream=None):
    arr = (C.c_int32 * len(precs))(*[PREC[p] if isinstance(p, str) else int(p) for p in precs])
    h = C.c_void_p()
    info = BucketInfo()
    _check(_lib.bspai_bucket(M.ptr, float(bucket_eps), arr, len(precs), _stream(stream), C.byref(h),
                             C.byref(info)))
    q = info.q
    d = dict(q=q, precs=[PREC_NAME[info.precs[k]] for k in range(q)], nnz_k=list(info.nnz_k[:q]),
             slots_k=list(info.slots_k[:q]), thresholds=list(info.thresholds[:q]), norm_inf=info.norm_inf,
             storage_pct=info.storage_pct, storage_pct_last8=info.storage_pct_last8, bytes=info.bytes)
    return BMHandle(h.value), d


def bucket_A(Ah: AHandle, bucket_eps: float, precs, stream=None):
    """Bucket A's own entries like M's (Section 3, eq. nbe2): row inf-norms of
    A, thresholds from bucket_eps, stored in the listed formats.  The handle
    works wherever a bucketed M does (apply, bucket_export) and as the A of
    gmres_b / gmres_ir_solve_hb."""
    arr = (C.c_int32 * len(precs))(*[PREC[p] if isinstance(p, str) else int(p) for p in precs])
    h = C.c_void_p()
    info = BucketInfo()
    _check(_lib.bspai_bucket_A(Ah.ptr, float(bucket_eps), arr, len(precs), _stream(stream), C.byref(h),
                               C.byref(info)))
    return BMHandle(h.value), _bucket_info(info)


def _bucket_info(info: BucketInfo) -> dict:
    q = info.q
    return dict(q=q, precs=[PREC_NAME[info.precs[k]] for k in range(q)], nnz_k=list(info.nnz_k[:q]),
                slots_k=list(info.slots_k[:q]), thresholds=list(info.thresholds[:q]), norm_inf=info.norm_inf,
                storage_pct=info.storage_pct, storage_pct_last8=info.storage_pct_last8, bytes=info.bytes)


def bspai_bucket_batched(M: MHandle, row_off, bucket_eps: float, precs, stream=None):
    """Per-system bucketing of a block-diagonal batch (row_off: device int32, nsys + 1)."""
    arr = (C.c_int32 * len(precs))(*[PREC[p] if isinstance(p, str) else int(p) for p in precs])
    h = C.c_void_p()
    info = BucketInfo()
    _check(_lib.bspai_bucket_batched(M.ptr, _ptr(row_off), int(row_off.numel() - 1), float(bucket_eps), arr,
                                     len(precs), _stream(stream), C.byref(h), C.byref(info)))
    return BMHandle(h.value), _bucket_info(info)


def bucket_export(BM: BMHandle, nnz: int, stream=None):
    ids = torch.empty(nnz, dtype=torch.int8, device="cuda")
    stored = torch.empty(nnz, dtype=torch.float64, device="cuda")
    _check(_lib.bspai_bucket_export(BM.ptr, _ptr(ids), _ptr(stored), _stream(stream)))
    return ids, stored


def apply(BM: BMHandle, x, y, stream=None):
    xp = PREC["fp64"] if x.dtype == torch.float64 else PREC["fp32"]
    yp = PREC["fp64"] if y.dtype == torch.float64 else PREC["fp32"]
    _check(_lib.bspai_apply(BM.ptr, _ptr(x), xp, _ptr(y), yp, _stream(stream)))
    return y


# ------------------------------------------------------------------ adjoint
def matrix_transpose(Ah: AHandle, stream=None) -> AHandle:
    h = C.c_void_p()
    _check(_lib.bspai_matrix_transpose(Ah.ptr, _stream(stream), C.byref(h)))
    return AHandle(h.value)


def M_transpose(M: MHandle, stream=None) -> MHandle:
    h = C.c_void_p()
    _check(_lib.bspai_M_transpose(M.ptr, _stream(stream), C.byref(h)))
    return MHandle(h.value)


def bucket_transpose(BM: BMHandle, stream=None) -> BMHandle:
    h = C.c_void_p()
    _check(_lib.bspai_bucket_transpose(BM.ptr, _stream(stream), C.byref(h)))
    return BMHandle(h.value)


def adjoint_grad_A(A: DeviceCSR, lam, x, dA, stream=None):
    """dA = sum over the right-hand sides r of -lambda_r[i] x_r[j] on A's
    nonzeros; lam and x: (n,) or (nrhs, n) contiguous fp64 device tensors."""
    nrhs = 1 if lam.dim() == 1 else int(lam.shape[0])
    assert x.shape == lam.shape and lam.is_contiguous() and x.is_contiguous()
    _check(_lib.bspai_adjoint_grad_A(C.byref(A.c()), nrhs, _ptr(lam), _ptr(x), _ptr(dA), _stream(stream)))
    return dA


# ------------------------------------------------------------------ solves
def _solve_info(si: SolveInfo) -> dict:
    k = si.ir_steps
    return dict(status=si.status, status_name=STATUS_NAMES[si.status], ir_steps=k, stop_reason=si.stop_reason,
                total_iters=si.total_iters, gmres_iters=list(si.gmres_iters[:k]),
                nbe=list(si.nbe[:min(33, k + 1)]), dx=list(si.dx[:k]), relres=list(si.relres[:k]), kmem=si.kmem,
                gmres_cycles=list(si.gmres_cycles[:k]))


def probe_fma(prec="fp32", iters=4096, stream=None) -> dict:
    """Measured lane-FMA rate of the plain fp32 / fp64 pipes (a measurement aid)."""
    r, ms = C.c_double(0.0), C.c_float(0.0)
    _check(_lib.bspai_probe_fma(PREC[prec], iters, _stream(stream), C.byref(r), C.byref(ms)))
    return dict(fma_per_s=r.value, flops=2.0 * r.value, ms=ms.value)


def apply_cw(M: MHandle, bucket_eps: float, precs, x, y, ids=None, counts=False, stream=None):
    """Componentwise, x-dependent bucketed product y = M x (bspai_apply_cw);
    returns the per-bucket counts when counts is set."""
    q = len(precs)
    arr = (C.c_int32 * q)(*[PREC[p] for p in precs])
    nk = (C.c_int64 * q)() if counts else None
    xp = PREC["fp64"] if x.dtype == torch.float64 else PREC["fp32"]
    yp = PREC["fp64"] if y.dtype == torch.float64 else PREC["fp32"]
    _check(_lib.bspai_apply_cw(M.ptr, bucket_eps, arr, q, _ptr(x), xp, _ptr(y), yp,
                               _ptr(ids) if ids is not None else None, nk, _stream(stream)))
    return list(nk) if counts else None


MGS_KERNELS = {0: "k_mgs", 1: "k_mgs_res", 2: "k_mgs_res2"}


def gmres_plan(n: int, u_g="fp32", max_blocks=0) -> dict:
    """The MGS kernel instance the GMRES solves pick for order n (a query)."""
    p = GmresPlan()
    _check(_lib.bspai_gmres_plan(n, PREC[u_g], max_blocks, C.byref(p)))
    return dict(kernel=MGS_KERNELS[p.kernel], per_thread=p.per_thread, block_threads=p.block_threads,
                blocks=p.blocks, poll="bulk" if p.poll_bulk else "loads")


def gmres(Ah: AHandle, BM: BMHandle, r, d, u_g="fp32", u_p="fp32", o: Opts | None = None, stream=None) -> dict:
    si = SolveInfo()
    st = _lib.bspai_gmres(Ah.ptr, BM.ptr, _ptr(r), PREC[u_g], PREC[u_p], C.byref(o or opts()), _ptr(d),
                          _stream(stream), C.byref(si))
    _check(st, (OK, NONFINITE))
    out = _solve_info(si)
    out["status"] = st
    return out


def gmres_b(Ah: AHandle, BA: BMHandle, BM: BMHandle, r, d, u_g="fp32", o: Opts | None = None,
            stream=None) -> dict:
    """bspai_gmres with A v taken through A's buckets (bucket_A) instead of A in u_p."""
    si = SolveInfo()
    st = _lib.bspai_gmres_b(Ah.ptr, BA.ptr, BM.ptr, _ptr(r), PREC[u_g], C.byref(o or opts()), _ptr(d),
                            _stream(stream), C.byref(si))
    _check(st, (OK, NONFINITE))
    out = _solve_info(si)
    out["status"] = st
    return out


def gmres_noalloc(Ah: AHandle, BM: BMHandle, r, d, u_g="fp32", u_p="fp32", o: Opts | None = None,
                  stream=None) -> dict:
    """bspai_gmres with its workspace in the library's fixed device block
    (for callers that cannot allocate device memory during the call)."""
    si = SolveInfo()
    st = _lib.bspai_gmres_noalloc(Ah.ptr, BM.ptr, _ptr(r), PREC[u_g], PREC[u_p], C.byref(o or opts()), _ptr(d),
                                  _stream(stream), C.byref(si))
    _check(st, (OK, NONFINITE))
    out = _solve_info(si)
    out["status"] = st
    return out


def gmres_ir_solve(A, b, BM: BMHandle, M: MHandle | None, x, u="fp64", u_r="dd", u_g="fp32", u_p="fp32",
                   tol=1e-4, o: Opts | None = None, stream=None) -> dict:
    """A: DeviceCSR (converted inside the call) or an AHandle from matrix_create."""
    si = SolveInfo()
    mp = M.ptr if M is not None else None
    if isinstance(A, AHandle):
        st = _lib.gmres_ir_solve_h(A.ptr, _ptr(b), BM.ptr, mp, PREC[u], PREC[u_r], PREC[u_g], PREC[u_p],
                                   float(tol), C.byref(o or opts()), _ptr(x), _stream(stream), C.byref(si))
    else:
        st = _lib.gmres_ir_solve(C.byref(A.c()), _ptr(b), BM.ptr, mp, PREC[u], PREC[u_r], PREC[u_g], PREC[u_p],
                                 float(tol), C.byref(o or opts()), _ptr(x), _stream(stream), C.byref(si))
    _check(st, (OK, NOT_CONVERGED, NONFINITE))
    out = _solve_info(si)
    out["status"] = st
    return out


def gmres_ir_solve_hb(Ah: AHandle, BA: BMHandle, b, BM: BMHandle, M: MHandle | None, x, u="fp64", u_r="dd",
                      u_g="fp32", tol=1e-4, o: Opts | None = None, stream=None) -> dict:
    """gmres_ir_solve with A v inside GMRES through A's buckets (bucket_A)."""
    si = SolveInfo()
    st = _lib.gmres_ir_solve_hb(Ah.ptr, BA.ptr, _ptr(b), BM.ptr, M.ptr if M is not None else None, PREC[u],
                                PREC[u_r], PREC[u_g], float(tol), C.byref(o or opts()), _ptr(x), _stream(stream),
                                C.byref(si))
    _check(st, (OK, NOT_CONVERGED, NONFINITE))
    out = _solve_info(si)
    out["status"] = st
    return out


def batch_schedule_force(block_threads: int | None = None, mgs_rows: int = 0, z_shared_rows: int = 0,
                         m_schedule: int = 0, team_rows: int = 0) -> None:
    """Fixes the schedule of this thread's later batched solves (block_threads
    None: back to the autotuner); see bspai_batch_schedule_t."""
    if block_threads is None:
        _check(_lib.bspai_batch_schedule_force(None))
        return
    sc = BatchSchedule(int(block_threads), int(mgs_rows), int(z_shared_rows), int(m_schedule), int(team_rows))
    _check(_lib.bspai_batch_schedule_force(C.byref(sc)))


def batch_tune_table() -> list[dict]:
    """The candidates the most recent batch autotuning timed, in order, with the
    GPU milliseconds of each one's sample run (the largest pairs, four per SM,
    32 Arnoldi steps)."""
    cnt = C.c_int32(0)
    _check(_lib.bspai_batch_tune_table(None, None, 0, C.byref(cnt)))
    n = cnt.value
    sc = (BatchSchedule * max(n, 1))()
    ms = (C.c_float * max(n, 1))()
    _check(_lib.bspai_batch_tune_table(sc, ms, n, C.byref(cnt)))
    return [dict(block_threads=sc[i].block_threads, mgs_rows=sc[i].mgs_rows, z_shared_rows=sc[i].z_shared_rows,
                 m_schedule=sc[i].m_schedule, team_rows=sc[i].team_rows, ms=float(ms[i]))
            for i in range(min(n, cnt.value))]


def gmres_ir_solve_batched(Ah: AHandle, row_off, nrhs: int, B, BM: BMHandle, M: MHandle | None, X, u_g="fp32",
                           u_p="fp32", tol=1e-4, o: Opts | None = None, pair_status=None, pair_iters=None,
                           stream=None) -> dict:
    """Batched BSPAI-GMRES-IR over block-diagonally stacked systems (row_off:
    device int32, nsys + 1; B, X: device fp64, nrhs * n)."""
    bi = BatchInfo()
    nsys = int(row_off.numel() - 1)
    st = _lib.gmres_ir_solve_batched(Ah.ptr, _ptr(row_off), nsys, int(nrhs), _ptr(B), BM.ptr,
                                     M.ptr if M is not None else None, PREC[u_g], PREC[u_p], float(tol),
                                     C.byref(o or opts()), _ptr(X), _stream(stream), C.byref(bi), _ptr(pair_status),
                                     _ptr(pair_iters))
    _check(st, (OK, NOT_CONVERGED, NONFINITE))
    d = {f: getattr(bi, f) for f, _ in BatchInfo._fields_}
    d["status"] = st
    return d
