"""Seeded synthetic inputs for BSPAI-GMRES-IR.

This module produces the matrices, sparsity patterns and right-hand sides
that both the CUDA path and the CPU oracle consume.  It holds none of the
method's arithmetic (no SPAI, bucketing, SpMV-in-precision, GMRES or
refinement); it only builds test problems shaped like the paper's workloads
(sparse nonsymmetric systems with a nonzero diagonal, Section 4 and Table 1)
plus the a-priori patterns named in Section 2.2 ("the sparsity pattern of A,
A^T, or a power of a sparsified A").

Everything is host-side numpy (CSR with int32 row pointers / columns and
float64 values, columns sorted ascending within each row).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

DEFAULT_SEED = 20230707


@dataclass
class CSR:
    """Host CSR matrix: ``row_ptr`` (n+1, int32), ``col`` (nnz, int32),
    ``val`` (nnz, float64 or None for a pure pattern)."""

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray | None

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        v = self.val if self.val is not None else np.ones(self.nnz)
        return sp.csr_matrix((v, self.col, self.row_ptr), shape=(self.n, self.n))

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def _from_dense_rows(cols: np.ndarray, vals: np.ndarray) -> CSR:
    """Pack an (n, w) table of columns (-1 = absent, ascending per row) into CSR."""
    mask = cols >= 0
    lens = mask.sum(axis=1)
    row_ptr = np.zeros(cols.shape[0] + 1, dtype=np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    return CSR(
        n=cols.shape[0],
        row_ptr=row_ptr.astype(np.int32),
        col=cols[mask].astype(np.int32),
        val=vals[mask].astype(np.float64),
    )


def convdiff2d(nx: int = 32, ny: int | None = None, peclet=(0.5, 0.5)) -> CSR:
    """2D convection-diffusion on an nx-by-ny interior grid with Dirichlet
    boundaries, 5-point centred stencil in dimensionless form: centre 4 and
    neighbours -1 -/+ P per direction (upwind side gets -(1+P)), wind along +x, +y.
    nx = ny = 32 gives n = 1024, nnz = 5n - 4*32 = 4992."""
    ny = nx if ny is None else ny
    px, py = peclet
    n = nx * ny
    r = np.arange(n, dtype=np.int64)
    ix, iy = r % nx, r // nx
    cols = np.full((n, 5), -1, dtype=np.int64)
    vals = np.zeros((n, 5))
    # ascending column order: south, west, centre, east, north
    cols[:, 0] = np.where(iy > 0, r - nx, -1)
    vals[:, 0] = -(1.0 + py)
    cols[:, 1] = np.where(ix > 0, r - 1, -1)
    vals[:, 1] = -(1.0 + px)
    cols[:, 2] = r
    vals[:, 2] = 4.0
    cols[:, 3] = np.where(ix < nx - 1, r + 1, -1)
    vals[:, 3] = -(1.0 - px)
    cols[:, 4] = np.where(iy < ny - 1, r + nx, -1)
    vals[:, 4] = -(1.0 - py)
    return _from_dense_rows(cols, vals)


def convdiff3d(g: int | tuple = 128, eps=(1.0, 10.0, 100.0), peclet: float = 0.8) -> CSR:
    """3D anisotropic convection-diffusion, 7-point stencil on a gx*gy*gz interior
    grid with Dirichlet boundaries.  Per direction d with diffusion eps_d and cell
    Peclet P: centre += 2 eps_d, lower neighbour -eps_d (1+P), upper -eps_d (1-P).
    g = 128 gives n = 2,097,152 and nnz = 7n - 6*128^2 = 14,581,760."""
    gx, gy, gz = (g, g, g) if np.isscalar(g) else g
    n = gx * gy * gz
    r = np.arange(n, dtype=np.int64)
    ix = r % gx
    iy = (r // gx) % gy
    iz = r // (gx * gy)
    ex, ey, ez = eps
    p = peclet
    cols = np.full((n, 7), -1, dtype=np.int64)
    vals = np.zeros((n, 7))
    sxy = gx * gy
    cols[:, 0] = np.where(iz > 0, r - sxy, -1)
    vals[:, 0] = -ez * (1 + p)
    cols[:, 1] = np.where(iy > 0, r - gx, -1)
    vals[:, 1] = -ey * (1 + p)
    cols[:, 2] = np.where(ix > 0, r - 1, -1)
    vals[:, 2] = -ex * (1 + p)
    cols[:, 3] = r
    vals[:, 3] = 2.0 * (ex + ey + ez)
    cols[:, 4] = np.where(ix < gx - 1, r + 1, -1)
    vals[:, 4] = -ex * (1 - p)
    cols[:, 5] = np.where(iy < gy - 1, r + gx, -1)
    vals[:, 5] = -ey * (1 - p)
    cols[:, 6] = np.where(iz < gz - 1, r + sxy, -1)
    vals[:, 6] = -ez * (1 - p)
    return _from_dense_rows(cols, vals)


# Diagonal factor of the random workload: with 1 + delta = 0.65 the diagonal no
# longer dominates its row and kappa_inf(A) ~ 5.3e5 at n = 65,536 (Hager-Higham
# estimate; found by oracle/condition_random.py, recorded in
# oracle/random_conditioning.json), in the 1e6 class of conditioning the
# random workload stands for.  delta >= 0 would keep kappa_inf near 1.6e4.
RANDOM_DELTA = -0.35


def random_sparse(n: int = 65536, k: int = 16, sigma: float = 2.0, delta: float = 1e-3,
                  seed: int = DEFAULT_SEED) -> CSR:
    """Random nonsymmetric sparse matrix: per row k distinct off-diagonal columns
    drawn uniformly, values sign * exp(N(0, sigma)), and a diagonal
    (1 + delta) * sum_j |a_ij|: strictly diagonally dominant for delta > 0;
    delta < 0 lowers the diagonal below the row sum and raises kappa_inf
    (delta controls the conditioning)."""
    rng = np.random.default_rng(seed)
    k = min(k, n - 1)
    cols = rng.integers(0, n - 1, size=(n, k), dtype=np.int64)
    rows = np.arange(n, dtype=np.int64)[:, None]
    while True:
        cols.sort(axis=1)
        dup = np.zeros(n, dtype=bool)
        dup |= (np.diff(cols, axis=1) == 0).any(axis=1)
        bad = np.nonzero(dup)[0]
        if bad.size == 0:
            break
        cols[bad] = rng.integers(0, n - 1, size=(bad.size, k), dtype=np.int64)
    # map [0, n-1) onto the off-diagonal columns of each row (skip the diagonal)
    cols = np.where(cols >= rows, cols + 1, cols)
    cols.sort(axis=1)
    mag = np.exp(rng.normal(0.0, sigma, size=(n, k)))
    sgn = np.where(rng.random((n, k)) < 0.5, -1.0, 1.0)
    off = sgn * mag
    diag = (1.0 + delta) * np.abs(off).sum(axis=1)
    allc = np.concatenate([cols, rows], axis=1)
    allv = np.concatenate([off, diag[:, None]], axis=1)
    order = np.argsort(allc, axis=1, kind="stable")
    allc = np.take_along_axis(allc, order, axis=1)
    allv = np.take_along_axis(allv, order, axis=1)
    return _from_dense_rows(allc, allv)


def lognormal_field(g: int, sigma: float = 1.0, corr: float = 8.0, seed: int = DEFAULT_SEED) -> np.ndarray:
    """kappa = exp(f) on a g x g grid, f a zero-mean Gaussian field with
    standard deviation sigma and squared-exponential correlation of length
    `corr` cells, made by filtering seeded white noise in Fourier space."""
    rng = np.random.default_rng(seed + 7)
    w = rng.normal(size=(g, g))
    k = np.fft.fftfreq(g)
    kx, ky = np.meshgrid(k, k, indexing="ij")
    filt = np.exp(-0.5 * (2 * np.pi) ** 2 * (kx ** 2 + ky ** 2) * corr ** 2 / 2.0)
    f = np.real(np.fft.ifft2(np.fft.fft2(w) * filt))
    f = (f - f.mean()) / f.std() * sigma
    return np.exp(f)


def diffusion2d(kappa: np.ndarray) -> CSR:
    """-div(kappa grad u) on the cell grid of `kappa` (g x g), Dirichlet u = 0
    outside, 5-point finite volumes: face coefficient = harmonic mean of the
    two cells' kappa (2 kappa_cell towards the boundary).  Symmetric, positive
    definite; rows ordered r = ix + g * iy."""
    g = kappa.shape[0]
    n = g * g
    kap = kappa.reshape(-1)  # index ix + g * iy with kappa[iy, ix]
    r = np.arange(n, dtype=np.int64)
    ix, iy = r % g, r // g

    def face(a, b):
        return 2.0 * a * b / (a + b)

    cols = np.full((n, 5), -1, dtype=np.int64)
    vals = np.zeros((n, 5))
    diag = np.zeros(n)
    nbrs = [(iy > 0, -g), (ix > 0, -1), (ix < g - 1, 1), (iy < g - 1, g)]
    slot = {-g: 0, -1: 1, 1: 3, g: 4}
    for ok, off in nbrs:
        j = np.where(ok, r + off, r)
        t = np.where(ok, face(kap, kap[j]), 2.0 * kap)
        diag += t
        cols[:, slot[off]] = np.where(ok, r + off, -1)
        vals[:, slot[off]] = -t
    cols[:, 2] = r
    vals[:, 2] = diag
    return _from_dense_rows(cols, vals)


def pattern_of(A: CSR) -> CSR:
    """The a-priori pattern pattern(A) (values dropped)."""
    return CSR(A.n, A.row_ptr.copy(), A.col.copy(), None)


def pattern_power_topk(A: CSR, keep: int = 24) -> CSR:
    """Pattern of |A|*|A| thinned to the `keep` largest entries per row,
    always keeping the diagonal, ties broken by the smaller column index.
    Row k of the result is the pattern of row k of M."""
    import scipy.sparse as sp

    S = abs(A.to_scipy())
    C = (S @ S).tocsr()
    C.sort_indices()
    n = A.n
    rp = C.indptr.astype(np.int64)
    cc = C.indices.astype(np.int64)
    vv = C.data.astype(np.float64).copy()
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    vv[cc == rows] = np.inf  # the diagonal is always kept
    order = np.lexsort((cc, -vv, rows))
    rank = np.empty_like(order)
    starts = np.repeat(rp[:-1], np.diff(rp))
    rank[order] = np.arange(order.size) - starts
    keepm = rank < keep
    kr, kc = rows[keepm], cc[keepm]
    o = np.lexsort((kc, kr))
    kr, kc = kr[o], kc[o]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, kr + 1, 1)
    np.cumsum(row_ptr, out=row_ptr)
    return CSR(n, row_ptr.astype(np.int32), kc.astype(np.int32), None)


def rhs(A: CSR, seed: int = DEFAULT_SEED, nrhs: int = 1):
    """x_true ~ U[-1, 1] (seeded) and b = A x_true in float64."""
    rng = np.random.default_rng(seed + 1)
    if nrhs == 1:
        x = rng.uniform(-1.0, 1.0, size=A.n)
    else:
        x = rng.uniform(-1.0, 1.0, size=(nrhs, A.n))
    As = A.to_scipy()
    b = (As @ x.T).T if nrhs > 1 else As @ x
    return x, np.ascontiguousarray(b)


def convdiff2d_9pt(g: int, peclet=(0.5, 0.5)) -> CSR:
    """2D 9-point compact Laplacian (centre 8, eight neighbours -1) plus centred
    convection on the four edge neighbours (-/+ P per direction, upwind side
    -(1+P)), g x g interior grid, Dirichlet boundaries."""
    px, py = peclet
    n = g * g
    r = np.arange(n, dtype=np.int64)
    ix, iy = r % g, r // g
    offs = [(-1, -1), (0, -1), (1, -1), (-1, 0), (0, 0), (1, 0), (-1, 1), (0, 1), (1, 1)]
    cols = np.full((n, 9), -1, dtype=np.int64)
    vals = np.zeros((n, 9))
    for k, (dx, dy) in enumerate(offs):  # ascending column order: row above, own row, row below
        ok = (ix + dx >= 0) & (ix + dx < g) & (iy + dy >= 0) & (iy + dy < g)
        cols[:, k] = np.where(ok, r + dx + g * dy, -1)
        v = 8.0 if (dx, dy) == (0, 0) else -1.0
        if (dx, dy) == (-1, 0):
            v = -(1.0 + px)
        elif (dx, dy) == (1, 0):
            v = -(1.0 - px)
        elif (dx, dy) == (0, -1):
            v = -(1.0 + py)
        elif (dx, dy) == (0, 1):
            v = -(1.0 - py)
        vals[:, k] = v
    return _from_dense_rows(cols, vals)


def block_diagonal(mats, align: int = 32):
    """Stack CSR matrices block-diagonally, each padded with empty rows to a
    multiple of `align` rows.  Returns (CSR, row_off) with row_off[s] the first
    row of system s (len nsys + 1)."""
    row_off = [0]
    for M in mats:
        row_off.append(row_off[-1] + -(-M.n // align) * align)
    n = row_off[-1]
    lens = np.zeros(n, dtype=np.int64)
    cols, vals = [], []
    for s, M in enumerate(mats):
        lens[row_off[s]:row_off[s] + M.n] = np.diff(M.row_ptr)
        cols.append(M.col.astype(np.int64) + row_off[s])
        if M.val is not None:
            vals.append(M.val)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    val = np.concatenate(vals) if vals else None
    return CSR(n, row_ptr.astype(np.int32), np.concatenate(cols).astype(np.int32), val), np.array(row_off, np.int32)


def batch_workload(nsys: int = 512, nrhs: int = 32, nmin: float = 1e3, nmax: float = 6.4e4,
                   seed: int = DEFAULT_SEED) -> dict:
    """Many independent 2D convection-diffusion systems: n = g^2 with
    g = round(sqrt(exp(U[ln nmin, ln nmax]))) (log-uniform sizes), a 5-point or
    9-point stencil with probability 1/2, cell Peclet ~ U[0.1, 1] per direction,
    pattern(A), nrhs right-hand sides b = A x_true with x_true ~ U[-1, 1].
    Systems are stacked block-diagonally (padded to multiples of 32 rows); B
    and X_true hold nrhs vectors of the stacked length."""
    rng = np.random.default_rng(seed + 11)
    mats, sizes = [], []
    for _ in range(nsys):
        g = int(round(np.sqrt(np.exp(rng.uniform(np.log(nmin), np.log(nmax))))))
        pe = tuple(rng.uniform(0.1, 1.0, 2))
        A = convdiff2d(g, g, pe) if rng.random() < 0.5 else convdiff2d_9pt(g, pe)
        mats.append(A)
        sizes.append(A.n)
    A, row_off = block_diagonal(mats)
    real = np.zeros(A.n, dtype=bool)
    for s, m in enumerate(mats):
        real[row_off[s]:row_off[s] + m.n] = True
    X = rng.uniform(-1.0, 1.0, size=(nrhs, A.n)) * real
    B = np.ascontiguousarray((A.to_scipy() @ X.T).T)
    return dict(name="batch", A=A, pattern=pattern_of(A), row_off=row_off, sizes=np.array(sizes), mats=mats,
                nrhs=nrhs, X_true=np.ascontiguousarray(X), B=B, real=real, spai_eps=0.3,
                precs=[FP64, FP32, FP16], bucket_eps=2.0 ** -16, tau=1e-4, u_g=FP32, u_p=FP32)


# ---------------------------------------------------------------------------
# Named workloads.  Each returns a dict with the matrix, the SPAI pattern and
# the solver settings of the workload; `scale` shrinks the grid for fast cases.
# ---------------------------------------------------------------------------

FP64, FP32, FP16, BF16, E4M3, DROP = "fp64", "fp32", "fp16", "bf16", "e4m3", "drop"


def workload(name: str, grid: int | None = None, n: int | None = None, seed: int = DEFAULT_SEED):
    """Named synthetic workloads.

    * ``convdiff2d``: 2D 5-point convection-diffusion, 32x32, Peclet 0.5,
      pattern(A), spai_eps 0.3, buckets {fp64, fp32, fp16}.
    * ``random``: random sparse n = 65,536, 16 off-diagonals per row, log-normal(0, 2),
      diagonal 0.65 times the row's sum (kappa_inf ~ 5e5), pattern(|A|^2) top-24,
      buckets {fp64, fp32, fp16, bf16}.
    * ``convdiff3d``: 3D 7-point anisotropic (1:10:100) convection-diffusion 128^3,
      Peclet 0.8, pattern(A), buckets {fp64, fp32, fp16, e4m3}.
    """
    if name == "convdiff2d":
        g = 32 if grid is None else grid
        A = convdiff2d(g, g, (0.5, 0.5))
        P = pattern_of(A)
        cfg = dict(spai_eps=0.3, precs=[FP64, FP32, FP16])
    elif name == "convdiff3d":
        g = 128 if grid is None else grid
        A = convdiff3d(g, (1.0, 10.0, 100.0), 0.8)
        P = pattern_of(A)
        cfg = dict(spai_eps=0.3, precs=[FP64, FP32, FP16, E4M3])
    elif name == "random":
        nn = 65536 if n is None else n
        A = random_sparse(nn, 16, 2.0, delta=RANDOM_DELTA, seed=seed)
        P = pattern_power_topk(A, 24)
        cfg = dict(spai_eps=0.3, precs=[FP64, FP32, FP16, BF16])
    elif name == "diffusion2d":
        g = 256 if grid is None else grid
        A = diffusion2d(lognormal_field(g, 1.0, 8.0, seed))
        P = pattern_of(A)
        cfg = dict(spai_eps=0.3, precs=[FP64, FP32, FP16])
    else:
        raise ValueError(f"unknown workload {name!r}")
    x_true, b = rhs(A, seed)
    cfg.update(bucket_eps=2.0 ** -37, u_f=FP32, u=FP64, u_r="dd", u_g=FP32, u_p=FP32, tau=1e-4)
    return dict(name=name, A=A, pattern=P, x_true=x_true, b=b, **cfg)
