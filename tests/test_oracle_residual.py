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
