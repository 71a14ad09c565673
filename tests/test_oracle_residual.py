"""Pins for the oracle's residual r = b - A x with u_r ~ u^2 (compensated dot
product Dot2; Alg 3.1 residual line)
against exact rational arithmetic."""
from fractions import Fraction

import numpy as np

from paper_2307_03914_gb300 import workloads as W


def _exact_residual(A, x, b):
    r = []
    for i in range(A.n):
        s = Fraction(b[i])
        for p in range(A.row_ptr[i], A.row_ptr[i + 1]):
            s -= Fraction(A.val[p]) * Fraction(x[A.col[p]])
        r.append(s)
    return r


def test_residual_dd_vs_exact_rational(orc):
    rng = np.random.default_rng(7)
    for trial in range(4):
        A = W.random_sparse(40, 6, sigma=3.0, delta=0.5, seed=100 + trial)
        x = rng.uniform(-1, 1, A.n) * np.exp(rng.normal(0, 4, A.n))
        # b close to A x so that the residual suffers heavy cancellation
        b = A.to_scipy() @ x
        b = b * (1 + rng.normal(0, 1e-13, A.n))
        r = orc.residual_dd(A, x, b)
        rex = _exact_residual(A, x, b)
        absax = abs(A.to_scipy()) @ np.abs(x) + np.abs(b)
        u = Fraction(1, 2 ** 53)
        for i in range(A.n):
            err = abs(Fraction(r[i]) - rex[i])
            # the Dot2 error bound (Ogita, Rump, Oishi 2005) for the n terms
            # b_i, -a_i1 x_1, ...: |res - r| <= u |r| + gamma_n^2 sum |terms|
            nt = int(A.row_ptr[i + 1] - A.row_ptr[i]) + 1
            gam = nt * u / (1 - nt * u)
            bound = u * abs(rex[i]) + gam * gam * Fraction(absax[i])
            assert err <= bound, (trial, i, float(err), float(bound))


def test_residual_dd_beats_fp64_on_cancellation(orc):
    # one row where fp64 evaluation loses everything but Dot2 does not
    A = W.CSR(1, np.array([0, 3], np.int32), np.array([0, 1, 2], np.int32),
              np.array([1.0, 1.0, 1.0]))
    x = np.array([1e16, 1.0, -1e16])
    b = np.array([0.0])
    r = orc.residual_dd(A, x, b)
    assert r[0] == -1.0  # exact: 0 - (1e16 + 1 - 1e16) = -1


def test_residual_fp64_textbook_bound_and_exact_integers(orc):
    """u_r = double: the plain recurrence obeys |r - exact| <= gamma_(p) (|b| +
    |A||x|) (Higham, Thm 3.5 read for b - sum a x), and is exact on small
    integer data (every intermediate is an integer below 2^53)."""
    rng = np.random.default_rng(9)
    for trial in range(4):
        A = W.random_sparse(40, 6, sigma=3.0, delta=0.5, seed=200 + trial)
        x = rng.uniform(-1, 1, A.n) * np.exp(rng.normal(0, 4, A.n))
        b = (A.to_scipy() @ x) * (1 + rng.normal(0, 1e-10, A.n))
        r = orc.residual_fp64(A, x, b)
        rex = _exact_residual(A, x, b)
        absax = abs(A.to_scipy()) @ np.abs(x) + np.abs(b)
        u = Fraction(1, 2 ** 53)
        worst = 0.0
        for i in range(A.n):
            p = int(A.row_ptr[i + 1] - A.row_ptr[i])
            gam = p * u / (1 - p * u)
            err = abs(Fraction(r[i]) - rex[i])
            assert err <= gam * Fraction(absax[i] * (1 + 2.0 ** -50)), (trial, i)
            worst = max(worst, float(err / Fraction(absax[i])))
        # the Dot2 residual is far more accurate on the same data
        rdd = orc.residual_dd(A, x, b)
        assert max(abs(Fraction(rdd[i]) - rex[i]) / Fraction(absax[i]) for i in range(A.n)) <= worst
    A = W.random_sparse(30, 5, sigma=1.0, delta=0.5, seed=9)
    Ai = W.CSR(A.n, A.row_ptr, A.col, np.round(A.val * 8))
    xi = rng.integers(-50, 50, A.n).astype(float)
    bi = rng.integers(-1000, 1000, A.n).astype(float)
    r = orc.residual_fp64(Ai, xi, bi)
    assert [Fraction(v) for v in r] == _exact_residual(Ai, xi, bi)
