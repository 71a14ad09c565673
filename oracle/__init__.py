"""CPU oracle for BSPAI-GMRES-IR (Khan & Carson, arXiv 2307.03914).

TEST INFRASTRUCTURE ONLY.  A plain, slow, obviously-sequential restatement of
the paper's algorithms (Alg 2.1 with a fixed pattern, Alg 2.2, Alg 2.3,
Alg 3.1) in C, wrapped here with ctypes and numpy.  Only the tests, the smoke
check and the benchmark's CPU-baseline leg import this package; the product
path never does, and the two share no code.

Parity status of each routine is recorded next to it below ("pinned by").
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bspai_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")

FMT = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3, "e4m3": 4, "drop": 5}
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp -ffp-contract=off)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(_SRC[:-2] + ".h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


class _System(C.Structure):
    _fields_ = [("n", C.c_int),
                ("arp", C.c_void_p), ("aci", C.c_void_p), ("av", C.c_void_p),
                ("mrp", C.c_void_p), ("mci", C.c_void_p), ("mstored", C.c_void_p),
                ("mid", C.c_void_p), ("fmts", C.c_void_p), ("q", C.c_int),
                ("astored", C.c_void_p), ("aid", C.c_void_p)]


def _declare(L):
    L.orc_fmt_bits.argtypes = [C.c_int]
    L.orc_fmt_bits.restype = C.c_int
    L.orc_unit_roundoff.argtypes = [C.c_int]
    L.orc_unit_roundoff.restype = C.c_double
    L.orc_fmt_max.argtypes = [C.c_int]
    L.orc_fmt_max.restype = C.c_double
    L.orc_round.argtypes = [C.c_double, C.c_int]
    L.orc_round.restype = C.c_double
    L.orc_round_array.argtypes = [_f64p, _f64p, C.c_int64, C.c_int]
    L.orc_set_threads.argtypes = [C.c_int]
    L.orc_get_threads.restype = C.c_int
    L.orc_residual_dd.argtypes = [C.c_int, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p]
    L.orc_residual_fp64.argtypes = [C.c_int, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p]
    L.orc_householder_ls.argtypes = [C.c_int, C.c_int, _f64p, _f64p, C.c_double, _f64p,
                                     C.POINTER(C.c_double)]
    L.orc_householder_ls.restype = C.c_int
    L.orc_row_absmax_scale.argtypes = [C.c_int, _i32p, _f64p, _f64p]
    L.orc_spai.argtypes = [C.c_int, _i32p, _i32p, _f64p, _i32p, _i32p, C.c_double, C.c_double,
                           C.c_int, C.c_int, _f64p, _f64p, _i32p, _i32p, _f64p]
    L.orc_spai.restype = C.c_int
    L.orc_spai_adaptive.argtypes = [C.c_int, _i32p, _i32p, _f64p, _i32p, _i32p, C.c_double, C.c_double,
                                    C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _i32p, _f64p,
                                    _i32p, _i8p, _f64p, _i32p, _i32p, _i32p, _i32p]
    L.orc_spai_adaptive.restype = C.c_int
    L.orc_spai_score.argtypes = [C.c_int, _i32p, _i32p, _f64p, _i32p, _i32p, _f64p, C.c_int, _i32p, C.c_int,
                                 C.c_double, C.c_int, C.c_int, _f64p, C.POINTER(C.c_double),
                                 C.POINTER(C.c_int), _i32p, _f64p, C.POINTER(C.c_int), C.POINTER(C.c_double),
                                 _i32p, C.POINTER(C.c_int)]
    L.orc_spai_score.restype = C.c_int
    L.orc_norm_inf.argtypes = [C.c_int, _i32p, _f64p]
    L.orc_norm_inf.restype = C.c_double
    L.orc_bucket_ids.argtypes = [C.c_int, _i32p, _f64p, C.c_double, _i32p, C.c_int, _i8p,
                                 _i64p, _f64p, C.POINTER(C.c_double)]
    L.orc_bucket_ids.restype = C.c_int
    L.orc_bucket_ids_cw.argtypes = [C.c_int, _i32p, _i32p, _f64p, _f64p, C.c_double, _i32p, C.c_int, _i8p,
                                    _i64p, _f64p]
    L.orc_bucket_ids_cw.restype = C.c_int
    L.orc_storage_pct.argtypes = [_i64p, _i32p, C.c_int, C.c_int]
    L.orc_storage_pct.restype = C.c_double
    L.orc_bucket_store.argtypes = [C.c_int, _i32p, _i32p, _f64p, _i8p, _i32p, C.c_int,
                                   _f64p, _f64p, _f64p]
    L.orc_bucket_store.restype = C.c_int
    L.orc_bspmv.argtypes = [C.c_int, _i32p, _i32p, _f64p, _i8p, _i32p, C.c_int, _f64p, _f64p]
    L.orc_bspmv_literal.argtypes = [C.c_int, _i32p, _i32p, _f64p, _i8p, _i32p, C.c_int,
                                    _f64p, _f64p]
    L.orc_spmv_prec.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_int, _f64p, _f64p]
    L.orc_gmres.argtypes = [C.POINTER(_System), _f64p, C.c_int, C.c_int, C.c_double, C.c_int,
                            _f64p, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.orc_gmres.restype = C.c_int
    L.orc_gmres_time_steps.argtypes = [C.c_void_p]
    L.orc_gmres_ir.argtypes = [C.POINTER(_System), _f64p, _f64p, C.c_int, C.c_int, C.c_double,
                               C.c_int, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, _f64p,
                               _i32p, _f64p, _f64p, C.POINTER(C.c_int)]
    L.orc_gmres_ir.restype = C.c_int
    L.orc_gmres_ir_m.argtypes = [C.POINTER(_System), _f64p, _f64p, C.c_int, C.c_int, C.c_double,
                                 C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int,
                                 _f64p, _i32p, _f64p, _f64p, C.POINTER(C.c_int), _i32p]
    L.orc_gmres_ir_m.restype = C.c_int
    L.orc_gmres_target.argtypes = [C.POINTER(_System), _f64p, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                                   _f64p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.POINTER(C.c_double)]
    L.orc_gmres_target.restype = C.c_int


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _fmts(fmts):
    return np.array([FMT[f] if isinstance(f, str) else int(f) for f in fmts], dtype=np.int32)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


# --------------------------------------------------------------- formats (O1)
def unit_roundoff(fmt) -> float:
    """Table 2 unit roundoffs.  Pinned by tests against the paper's printed values."""
    return lib().orc_unit_roundoff(FMT[fmt])


def fmt_bits(fmt) -> int:
    return lib().orc_fmt_bits(FMT[fmt])


def round_to(x, fmt) -> np.ndarray:
    """RN-even into `fmt` with its own range.  Pinned by exhaustive comparison
    against library casts (numpy/torch) in tests."""
    x = _f64(np.atleast_1d(x))
    y = np.empty_like(x)
    lib().orc_round_array(x, y, x.size, FMT[fmt])
    return y


# -------------------------------------------------------------- residual (O2)
def residual_dd(A, x, b) -> np.ndarray:
    """r = b - A x by the compensated dot product Dot2 (as accurate as a sum in
    twice fp64), rounded to fp64.  Pinned by exact rational
    arithmetic (fractions) in tests."""
    r = np.empty(A.n)
    lib().orc_residual_dd(A.n, _i32(A.row_ptr), _i32(A.col), _f64(A.val), _f64(x), _f64(b), r)
    return r


def residual_fp64(A, x, b) -> np.ndarray:
    """r = b - A x in plain fp64 (u_r = double), products and differences
    rounded in ascending column order.  Pinned by exact rational arithmetic
    (the textbook bound gamma_p (|b| + |A||x|)) and by exactness on integer data."""
    r = np.empty(A.n)
    lib().orc_residual_fp64(A.n, _i32(A.row_ptr), _i32(A.col), _f64(A.val), _f64(x), _f64(b), r)
    return r


# ------------------------------------------------------------------ SPAI (O3, O4)
def householder_ls(Ad: np.ndarray, b: np.ndarray, rank_tol: float = 0.0):
    """Dense Householder least squares.  Pinned against LAPACK (numpy.linalg.lstsq)."""
    m, k = Ad.shape
    x = np.zeros(k)
    res = C.c_double(0.0)
    rd = lib().orc_householder_ls(m, k, _f64(np.asfortranarray(Ad).ravel(order="F")), _f64(b),
                                  rank_tol, x, C.byref(res))
    return x, res.value, rd


def row_absmax_scale(A) -> np.ndarray:
    d = np.empty(A.n)
    lib().orc_row_absmax_scale(A.n, _i32(A.row_ptr), _f64(A.val), d)
    return d


def spai(A, P, spai_eps: float, u_f: float = 2.0 ** -24, cols=None) -> dict:
    """Fixed-pattern SPAI on A^T D, returning M = M'^T D in P's structure.
    Pinned by LAPACK lstsq, normal equations, M = A^-1 for a full pattern."""
    c0, c1 = (0, A.n) if cols is None else cols
    mval = np.zeros(P.nnz)
    resid = np.zeros(A.n)
    conv = np.zeros(A.n, dtype=np.int32)
    rankdef = np.zeros(A.n, dtype=np.int32)
    kappa = np.zeros(A.n)
    nbad = lib().orc_spai(A.n, _i32(A.row_ptr), _i32(A.col), _f64(A.val), _i32(P.row_ptr),
                          _i32(P.col), spai_eps, u_f, c0, c1, mval, resid, conv, rankdef, kappa)
    return dict(mval=mval, resid=resid, conv=conv, rankdef=rankdef, kappa=kappa, nbad=nbad)


def spai_adaptive(A, spai_eps: float, alpha: int, beta: int = 8, u_f: float = 2.0 ** -24,
                  imax_rows: int = 256, cap=None, cols=None) -> dict:
    """Adaptive SPAI (Alg 2.1, alpha > 0, Grote-Huckle growth) on A^T D from
    the identity pattern; M = M'^T D as CSR (row k = the final pattern J_k of
    column k of M').  Pinned by dense least squares on the pattern it returns,
    the 1-D minimisation behind rho (Section 2.2), the selection rule, the
    monotone residual, and M = A^-1 once the pattern fills a small matrix."""
    n = A.n
    cap = 1 + alpha * beta if cap is None else cap
    c0, c1 = (0, n) if cols is None else cols
    trp, tci, _ = transpose_csr(A.row_ptr, A.col, np.ones(A.nnz))
    Jo = np.full(n * cap, -1, dtype=np.int32)
    mo = np.zeros(n * cap)
    nJ = np.zeros(n, dtype=np.int32)
    st = np.zeros(n * cap, dtype=np.int8)
    resid = np.zeros(n)
    conv = np.zeros(n, dtype=np.int32)
    rankdef = np.zeros(n, dtype=np.int32)
    nsolves = np.zeros(n, dtype=np.int32)
    capped = np.zeros(n, dtype=np.int32)
    nbad = lib().orc_spai_adaptive(n, _i32(A.row_ptr), _i32(A.col), _f64(A.val), _i32(trp), _i32(tci), spai_eps,
                                   u_f, int(alpha), int(beta), int(imax_rows), c0, c1, int(cap), Jo, mo, nJ, st,
                                   resid, conv, rankdef, nsolves, capped)
    rows = np.arange(c0, c1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(nJ)
    sel = (np.arange(cap)[None, :] < nJ[:, None]).ravel()
    return dict(row_ptr=row_ptr.astype(np.int32), col=Jo[sel], mval=mo[sel], step_added=st[sel], nJ=nJ,
                resid=resid, conv=conv, rankdef=rankdef, nsolves=nsolves, capped=capped, nbad=nbad, rows=rows)


_SCORE_MEMO: dict = {}


def spai_score(A, k: int, J, beta: int = 8, u_f: float = 2.0 ** -24) -> dict:
    """One scoring pass of the adaptive SPAI for column k with pattern J."""
    key = (id(A), A.n, A.nnz)
    if key not in _SCORE_MEMO:  # A^T's structure and the scaling, once per matrix
        trp_, tci_, _ = transpose_csr(A.row_ptr, A.col, np.ones(A.nnz))
        _SCORE_MEMO.clear()
        _SCORE_MEMO[key] = (A, trp_, tci_, row_absmax_scale(A))
    _, trp, tci, d = _SCORE_MEMO[key]
    J = np.ascontiguousarray(np.sort(np.asarray(J)), dtype=np.int32)
    room = int(np.diff(trp).sum()) + 1
    mbar = np.zeros(max(len(J), 1))
    cand = np.zeros(room, dtype=np.int32)
    rho = np.zeros(room)
    picks = np.zeros(max(beta, 1), dtype=np.int32)
    sres, mean = C.c_double(0.0), C.c_double(0.0)
    rd, nc, npk = C.c_int(0), C.c_int(0), C.c_int(0)
    nI = lib().orc_spai_score(A.n, _i32(A.row_ptr), _i32(A.col), _f64(A.val), _i32(trp), _i32(tci), d, int(k), J,
                              len(J), u_f, int(beta), 1, mbar, C.byref(sres), C.byref(rd), cand, rho, C.byref(nc),
                              C.byref(mean), picks, C.byref(npk))
    return dict(nI=nI, mbar=mbar[:len(J)], sres=sres.value, rd=rd.value, cand=cand[:nc.value], rho=rho[:nc.value],
                mean=mean.value, picks=picks[:npk.value])


# ------------------------------------------------------------- bucketing (O5)
def norm_inf(row_ptr, val) -> float:
    return lib().orc_norm_inf(len(row_ptr) - 1, _i32(row_ptr), _f64(val))


def bucket_ids(row_ptr, val, bucket_eps: float, fmts) -> dict:
    """eq. (nint) / Alg 2.2.  Pinned by the Table 3 storage figures, hand-worked
    cases and the Graillat et al. backward-error bound (tests)."""
    f = _fmts(fmts)
    q = len(f)
    nnz = int(row_ptr[-1])
    ids = np.zeros(nnz, dtype=np.int8)
    nnz_k = np.zeros(q, dtype=np.int64)
    thr = np.zeros(q)
    nrm = C.c_double(0.0)
    rc = lib().orc_bucket_ids(len(row_ptr) - 1, _i32(row_ptr), _f64(val), bucket_eps, f, q, ids,
                              nnz_k, thr, C.byref(nrm))
    if rc != 0:
        raise ValueError("bucket precisions must have strictly increasing unit roundoff")
    return dict(ids=ids, nnz_k=nnz_k, thr=thr, norm=nrm.value)


def bucket_ids_cw(row_ptr, col, val, x, bucket_eps: float, fmts) -> dict:
    """Componentwise, x-dependent bucketing (Section 2.3 mentions it; reading:
    eq. (nint) on |a_ij| |x_j| against eps (|A||x|)_i / u_k, row by row).
    Pinned by the interval definition entry by entry and by the componentwise
    backward-error bound with exact rationals (tests)."""
    f = _fmts(fmts)
    q = len(f)
    n = len(row_ptr) - 1
    ids = np.zeros(int(row_ptr[-1]), dtype=np.int8)
    nnz_k = np.zeros(q, dtype=np.int64)
    srow = np.zeros(n)
    rc = lib().orc_bucket_ids_cw(n, _i32(row_ptr), _i32(col), _f64(val), _f64(x), bucket_eps, f, q, ids, nnz_k,
                                 srow)
    if rc != 0:
        raise ValueError("bucket precisions must have strictly increasing unit roundoff")
    return dict(ids=ids, nnz_k=nnz_k, srow=srow)


def storage_pct(nnz_k, fmts, last_bits: int = 0) -> float:
    f = _fmts(fmts)
    return lib().orc_storage_pct(np.ascontiguousarray(nnz_k, dtype=np.int64), f, len(f), last_bits)


def bucket_store(row_ptr, col, val, ids, fmts):
    f = _fmts(fmts)
    n = len(row_ptr) - 1
    stored = np.zeros(len(val))
    bscale = np.zeros(len(f))
    cscale = np.zeros(n)
    lib().orc_bucket_store(n, _i32(row_ptr), _i32(col), _f64(val), np.ascontiguousarray(ids, np.int8),
                           f, len(f), stored, bscale, cscale)
    return stored, bscale, cscale


# ------------------------------------------------------------------ SpMV (O6)
def bspmv(row_ptr, col, stored, ids, fmts, x) -> np.ndarray:
    """Alg 2.3, decoupled storage/compute form."""
    f = _fmts(fmts)
    n = len(row_ptr) - 1
    y = np.empty(n)
    lib().orc_bspmv(n, _i32(row_ptr), _i32(col), _f64(stored), np.ascontiguousarray(ids, np.int8),
                    f, len(f), _f64(x), y)
    return y


def bspmv_literal(row_ptr, col, val, ids, fmts, x) -> np.ndarray:
    """Alg 2.3 as printed: each bucket in its own precision and range."""
    f = _fmts(fmts)
    n = len(row_ptr) - 1
    y = np.empty(n)
    lib().orc_bspmv_literal(n, _i32(row_ptr), _i32(col), _f64(val),
                            np.ascontiguousarray(ids, np.int8), f, len(f), _f64(x), y)
    return y


def spmv_prec(row_ptr, col, val, fmt, x) -> np.ndarray:
    n = len(row_ptr) - 1
    y = np.empty(n)
    lib().orc_spmv_prec(n, _i32(row_ptr), _i32(col), _f64(val), FMT[fmt], _f64(x), y)
    return y


# ----------------------------------------------------------- GMRES / IR (O7, O8)
class System:
    """A together with a bucketed M (structure, stored values, bucket ids), and
    optionally A's own buckets (stored values and ids on A's pattern, same
    formats) for A v by the bucketed SpMV (eq. nbe2)."""

    def __init__(self, A, M_row_ptr, M_col, M_stored, M_ids, fmts, A_stored=None, A_ids=None):
        self._keep = [_i32(A.row_ptr), _i32(A.col), _f64(A.val), _i32(M_row_ptr), _i32(M_col),
                      _f64(M_stored), np.ascontiguousarray(M_ids, np.int8), _fmts(fmts)]
        k = self._keep
        astored = aid = None
        if A_stored is not None:
            self._keep += [_f64(A_stored), np.ascontiguousarray(A_ids, np.int8)]
            astored, aid = self._keep[8].ctypes.data, self._keep[9].ctypes.data
        self.n = A.n
        self.s = _System(A.n, k[0].ctypes.data, k[1].ctypes.data, k[2].ctypes.data,
                         k[3].ctypes.data, k[4].ctypes.data, k[5].ctypes.data, k[6].ctypes.data,
                         k[7].ctypes.data, len(k[7]), astored, aid)


def gmres(system: System, r, ug="fp32", up="fp32", tau=1e-4, kmax=500, step_seconds=False):
    """GMRES on (M A) d = M r (Alg 3.1, GMRES line): (d, iterations, |g_k|/beta),
    plus the wall time of every Arnoldi step when step_seconds is set (a
    measurement aid for the CPU baseline; the results are the same)."""
    d = np.zeros(system.n)
    it = C.c_int(0)
    rr = C.c_double(0.0)
    L = lib()
    ts = np.zeros(max(int(kmax), 1))
    if step_seconds:  # the timing pointer is one per library: one timed call at a time
        with _lock:
            L.orc_gmres_time_steps(ts.ctypes.data)
            L.orc_gmres(C.byref(system.s), _f64(r), FMT[ug], FMT[up], tau, int(kmax), d,
                        C.byref(it), C.byref(rr))
    else:
        L.orc_gmres(C.byref(system.s), _f64(r), FMT[ug], FMT[up], tau, int(kmax), d,
                    C.byref(it), C.byref(rr))
    if step_seconds:
        return d, it.value, rr.value, ts[:it.value].copy()
    return d, it.value, rr.value


UNIT_ROUNDOFF = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24}


def gmres_target(system: System, r, target, ug="fp32", up="fp32", tau=1e-4, kmax=500):
    """GMRES on (M A) d = M r stopping at |g_{j+1}| <= target (target > 0) instead
    of the tau test: (d, iterations, beta = ||M r||_2 in u_g, last |g|)."""
    d = np.zeros(system.n)
    it = C.c_int(0)
    rr, be, rs = C.c_double(0.0), C.c_double(0.0), C.c_double(0.0)
    lib().orc_gmres_target(C.byref(system.s), _f64(r), FMT[ug], FMT[up], tau, float(target), int(kmax), d,
                           C.byref(it), C.byref(rr), C.byref(be), C.byref(rs))
    return d, it.value, be.value, rs.value


def gmres_ir(system: System, muf, b, ug="fp32", up="fp32", tau=1e-4, kmax=500, imax=10,
             u_work=None, x0=None, u="fp64", u_r="dd", u_f="fp32", kmem=0) -> dict:
    """Alg 3.1 with working precision u (fp64, or fp32 for the (single,
    single, double) and (half, single, double) settings of Section 4) and
    residual precision u_r ("dd": Dot2, about twice fp64; "fp64": plain fp64).
    x0 = M b is taken in u_f arithmetic (fp32, or fp16 with its own range) on
    the values muf, which the caller holds in u_f.  x, r and the correction
    are held in u; u_work (the stopping level) defaults to u's unit roundoff."""
    if u not in UNIT_ROUNDOFF or u_r not in ("dd", "fp64"):
        raise ValueError("u must be fp64 or fp32, u_r dd or fp64")
    if u_f not in ("fp32", "fp16"):
        raise ValueError("u_f must be fp32 or fp16")
    u_work = UNIT_ROUNDOFF[u] if u_work is None else u_work
    x = np.zeros(system.n) if x0 is None else _f64(x0).copy()
    its = np.zeros(imax, dtype=np.int32)
    cyc = np.zeros(imax, dtype=np.int32)
    nbe = np.zeros(imax)
    dx = np.zeros(imax)
    stop = C.c_int(0)
    # kmem > 0: the Krylov basis capped at kmem + 1 vectors, each correction
    # equation solved by restarted GMRES cycles (orc_gmres_ir_m)
    steps = lib().orc_gmres_ir_m(C.byref(system.s), _f64(muf), _f64(b), FMT[ug], FMT[up], tau,
                                 int(kmax), int(kmem), int(imax), u_work, FMT[u], int(u_r == "dd"), FMT[u_f],
                                 int(x0 is not None), x, its, nbe, dx, C.byref(stop), cyc)
    nsteps = min(imax, steps + (1 if stop.value == 1 else 0))
    return dict(x=x, steps=steps, its=its[:max(steps, 0)].tolist(), nbe=nbe[:nsteps].tolist(),
                dx=dx[:steps].tolist(), stop=stop.value, cycles=cyc[:max(steps, 0)].tolist())


def transpose_csr(row_ptr, col, val):
    """CSR of the transpose (columns ascending), via scipy."""
    import scipy.sparse as sp

    n = len(row_ptr) - 1
    T = sp.csr_matrix((np.asarray(val, np.float64), np.asarray(col), np.asarray(row_ptr)), shape=(n, n)).T.tocsr()
    T.sort_indices()
    return T.indptr.astype(np.int32), T.indices.astype(np.int32), T.data.astype(np.float64)


class _Csr:
    def __init__(self, n, row_ptr, col, val):
        self.n, self.row_ptr, self.col, self.val = n, row_ptr, col, val


def adjoint(A, P, muf, x, g, kmax=500, imax=10, kmem=0) -> dict:
    """Adjoint of x = A^-1 b for a loss with dL/dx = g: lambda = A^-T g by the
    refinement driver in fp64 (u_g = u_p = fp64, tau = 1e-12) on A^T, left-
    preconditioned by M^T (q = 1, fp64); dL/db = lambda and dL/dA_ij =
    -lambda_i x_j on the nonzeros of A.  Pinned by dense solves and central
    finite differences (tests)."""
    trp, tcol, tval = transpose_csr(A.row_ptr, A.col, A.val)
    mrp, mcol, mval = transpose_csr(P.row_ptr, P.col, muf)
    At = _Csr(A.n, trp, tcol, tval)
    S = System(At, mrp, mcol, mval, np.zeros(len(mval), np.int8), ["fp64"])
    out = gmres_ir(S, mval, g, "fp64", "fp64", 1e-12, kmax, imax, kmem=kmem)
    lam = out["x"]
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    dA = -lam[rows] * np.asarray(x)[A.col]
    return dict(lam=lam, dA=dA, db=lam, info=out)


def adjoint_grad_A(A, lam, x) -> np.ndarray:
    """dL/dA_ij = -sum_r lam_r[i] x_r[j] on the nonzeros of A (CSR order) for
    nrhs right-hand sides, A x_r = b_r and lam_r = A^-T dL/dx_r (the adjoint
    extension; the gradient of a sum of losses is the sum of gradients).  The
    sum runs over r ascending from 0, every product and sum one fp64 rounding.
    lam, x: (n,) or (nrhs, n).  Pinned: nrhs = 1 is -lam_i x_j itself; on
    integer-valued inputs the sum is exact and equals Python's integer sum
    (tests)."""
    lam = np.atleast_2d(np.asarray(lam, np.float64))
    x = np.atleast_2d(np.asarray(x, np.float64))
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    acc = np.zeros(len(A.col))
    for r in range(lam.shape[0]):
        acc = acc + (-lam[r][rows]) * x[r][np.asarray(A.col)]
    return acc


def solve(wl: dict, bucket_eps=None, precs=None, kmax=500, imax=10, tau=None, bucket_A=False, u="fp64",
          u_r="dd", ug=None, up=None, adaptive=None, u_f="fp32", kmem=0) -> dict:
    """Full oracle pipeline on a workload dict: SPAI -> bucketing -> GMRES-IR.
    bucket_A: A v inside GMRES by the bucketed SpMV on A's own buckets (same
    precisions and bucket_eps, thresholds from ||A||_inf; eq. nbe2).
    adaptive: build M by the adaptive SPAI (spai_adaptive's keyword arguments)
    instead of on the workload's fixed pattern."""
    A, P = wl["A"], wl["pattern"]
    if adaptive is None:
        sp = spai(A, P, wl["spai_eps"])
    else:  # adaptive: dict(spai_eps, alpha, beta[, imax_rows]) -- Alg 2.1 from the identity pattern
        sp = spai_adaptive(A, **adaptive)
        P = _Csr(A.n, sp["row_ptr"], sp["col"], None)
    muf = round_to(sp["mval"], u_f)  # M is held in u_f (fp32, or fp16 for the (half, single, double) setting)
    precs = wl["precs"] if precs is None else precs
    be = wl["bucket_eps"] if bucket_eps is None else bucket_eps
    bk = bucket_ids(P.row_ptr, muf, be, precs)
    stored, _, _ = bucket_store(P.row_ptr, P.col, muf, bk["ids"], precs)
    a_stored = a_ids = None
    if bucket_A:
        ak = bucket_ids(A.row_ptr, A.val, be, precs)
        a_ids = ak["ids"]
        a_stored, _, _ = bucket_store(A.row_ptr, A.col, A.val, a_ids, precs)
    S = System(A, P.row_ptr, P.col, stored, bk["ids"], precs, a_stored, a_ids)
    out = gmres_ir(S, muf, wl["b"], wl["u_g"] if ug is None else ug, wl["u_p"] if up is None else up,
                   wl["tau"] if tau is None else tau, kmax, imax, u=u, u_r=u_r, u_f=u_f, kmem=kmem)
    out.update(spai=sp, muf=muf, buckets=bk, stored=stored)
    return out
