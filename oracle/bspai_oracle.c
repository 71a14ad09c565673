/*
 * bspai_oracle.c -- CPU oracle for BSPAI-GMRES-IR (Khan & Carson, arXiv 2307.03914).
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow restatement of the paper's
 * algorithms that the tests, the smoke check and the benchmark's CPU
 * baseline use to check and time the CUDA path.  Nothing in the product path
 * calls it.  No code is shared with the CUDA library.
 *
 * Section map:
 *   formats      Table 2 precisions; RN-even rounding written from the
 *                definition (round x / 2^(e-t+1) to an integer), as in the
 *                chop approach the paper uses for half precision (Section 4).
 *   residual     Alg 3.1 residual line with u_r ~ u^2: compensated dot
 *                product Dot2 (Knuth TwoSum, FMA TwoProduct; Ogita, Rump,
 *                Oishi 2005).
 *   SPAI         eq. (fronormmin), eq. (redprob), Alg 2.1 with alpha = 0;
 *                Householder QR (Golub & Van Loan Alg 5.2.1 sign choice);
 *                column scaling of Section 4.
 *   bucketing    eq. (nint) and Alg 2.2; storage cost of Tables 3/4.
 *   SpMV         Alg 2.3, in the decoupled storage/compute form (Section 5
 *                future work) and in the literal form.
 *   GMRES / IR   Alg 3.1: left-preconditioned MGS-GMRES with Givens
 *                rotations (Saad, Alg 6.9), refinement in u = fp64.
 *
 * Parity notes: every SpMV and the residual accumulate sequentially in
 * ascending column order; OpenMP only splits independent rows or columns,
 * so results do not depend on the thread count.
 */
#include "bspai_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ formats */

typedef struct { int t; int emin; double maxv; int sat; int bits; } fmt_t;

static fmt_t fmt_info(int f) {
    fmt_t r;
    switch (f) {
    case ORC_FP64: r.t = 53; r.emin = -1022; r.maxv = DBL_MAX; r.sat = 0; r.bits = 64; break;
    case ORC_FP32: r.t = 24; r.emin = -126; r.maxv = ldexp(2.0 - ldexp(1.0, -23), 127); r.sat = 0; r.bits = 32; break;
    case ORC_FP16: r.t = 11; r.emin = -14; r.maxv = 65504.0; r.sat = 0; r.bits = 16; break;
    case ORC_BF16: r.t = 8; r.emin = -126; r.maxv = ldexp(2.0 - ldexp(1.0, -7), 127); r.sat = 0; r.bits = 16; break;
    case ORC_E4M3: r.t = 4; r.emin = -6; r.maxv = 448.0; r.sat = 1; r.bits = 8; break;
    default: r.t = 0; r.emin = 0; r.maxv = 0.0; r.sat = 0; r.bits = 0; break; /* drop */
    }
    return r;
}

int orc_fmt_bits(int f) { return fmt_info(f).bits; }

double orc_unit_roundoff(int f) {
    if (f == ORC_DROP) return 1.0;
    return ldexp(1.0, -fmt_info(f).t);
}

double orc_fmt_max(int f) { return fmt_info(f).maxv; }

double orc_round(double x, int f) {
    if (f == ORC_FP64) return x;
    if (f == ORC_DROP) return 0.0;
    fmt_t F = fmt_info(f);
    if (x != x) return x;
    if (isinf(x)) return F.sat ? copysign(F.maxv, x) : x;
    if (x == 0.0) return x;
    int E;
    frexp(fabs(x), &E);        /* |x| = m 2^E, m in [0.5, 1): binade exponent E - 1 */
    int e = E - 1;
    if (e < F.emin) e = F.emin; /* subnormal range: fixed quantum */
    double quantum = ldexp(1.0, e - F.t + 1);
    double y = nearbyint(x / quantum) * quantum; /* default mode: ties to even */
    if (fabs(y) > F.maxv) y = F.sat ? copysign(F.maxv, x) : copysign(INFINITY, x);
    return y;
}

void orc_round_array(const double* x, double* y, int64_t n, int f) {
    for (int64_t i = 0; i < n; ++i) y[i] = orc_round(x[i], f);
}

void orc_set_threads(int nt) {
#ifdef _OPENMP
    if (nt > 0) omp_set_num_threads(nt);
#else
    (void)nt;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* emulated arithmetic in format f: one fp64 op, one rounding */
static inline double rf(double x, int f) { return f == ORC_FP64 ? x : orc_round(x, f); }

/* ------------------------------------------------ error-free transformations */

static inline void two_sum(double a, double b, double* s, double* e) {
    double S = a + b;
    double bv = S - a;
    *e = (a - (S - bv)) + (b - bv);
    *s = S;
}

static inline void two_prod(double a, double b, double* p, double* e) {
    double P = a * b;
    *e = fma(a, b, -P);
    *p = P;
}

/* r_i = b_i - sum_j a_ij x_j by Dot2 (Ogita, Rump and Oishi, "Accurate sum and
 * dot product", 2005): every product split exactly (TwoProduct by FMA), the
 * running sum p updated by TwoSum, the running error s collecting the TwoSum
 * errors and the products' errors, r_i = fl(p + s); ascending column order.
 * The result is as accurate as a sum in twice the working precision:
 * |r_i - exact| <= u |exact| + gamma_n^2 sum |terms|, so u_r ~ u^2 (Alg 3.1
 * residual line, with quad read as "at least twice fp64"). */
void orc_residual_dd(int n, const int* rp, const int* ci, const double* av,
                     const double* x, const double* b, double* r) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double p = b[i], s = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            double ph, pl, q;
            two_prod(av[k], x[ci[k]], &ph, &pl);
            two_sum(p, -ph, &p, &q);
            s = s + (q - pl);
        }
        r[i] = p + s;
    }
}

/* r = b - A x in plain fp64: r_i = (...((b_i - a_i1 x_1) - a_i2 x_2) ...), every
 * product and every difference rounded to fp64, ascending column order (Alg 3.1
 * residual line with u_r = double, the (single, single, double) setting of
 * Section 4). */
void orc_residual_fp64(int n, const int* rp, const int* ci, const double* av,
                       const double* x, const double* b, double* r) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double acc = b[i];
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            double p = av[k] * x[ci[k]];
            acc = acc - p;
        }
        r[i] = acc;
    }
}

/* ----------------------------------------------------------- Householder LS */

int orc_householder_ls(int m, int k, const double* A0, const double* b0, double rank_tol,
                       double* x, double* resid) {
    double* A = (double*)malloc(sizeof(double) * (size_t)m * (size_t)k);
    double* c = (double*)malloc(sizeof(double) * (size_t)m);
    double* v = (double*)malloc(sizeof(double) * (size_t)m);
    memcpy(A, A0, sizeof(double) * (size_t)m * (size_t)k);
    memcpy(c, b0, sizeof(double) * (size_t)m);
    int deficient = 0;
    for (int j = 0; j < k; ++j) {
        /* reflector annihilating A(j+1:m, j) */
        double sig = 0.0;
        for (int i = j; i < m; ++i) sig += A[(size_t)j * m + i] * A[(size_t)j * m + i];
        sig = sqrt(sig);
        double x0 = A[(size_t)j * m + j];
        if (sig == 0.0) { deficient = 1; continue; }
        double sgn = x0 >= 0.0 ? 1.0 : -1.0;
        for (int i = j; i < m; ++i) v[i] = A[(size_t)j * m + i];
        v[j] = x0 + sgn * sig;
        double vtv = 0.0;
        for (int i = j; i < m; ++i) vtv += v[i] * v[i];
        for (int jj = j; jj < k; ++jj) {
            double dot = 0.0;
            for (int i = j; i < m; ++i) dot += v[i] * A[(size_t)jj * m + i];
            double tau = 2.0 * dot / vtv;
            for (int i = j; i < m; ++i) A[(size_t)jj * m + i] -= tau * v[i];
        }
        double dot = 0.0;
        for (int i = j; i < m; ++i) dot += v[i] * c[i];
        double tau = 2.0 * dot / vtv;
        for (int i = j; i < m; ++i) c[i] -= tau * v[i];
        A[(size_t)j * m + j] = -sgn * sig; /* R_jj */
    }
    for (int j = 0; j < k; ++j)
        if (!(fabs(A[(size_t)j * m + j]) > rank_tol)) deficient = 1;
    if (deficient) {
        for (int j = 0; j < k; ++j) x[j] = 0.0;
    } else {
        for (int j = k - 1; j >= 0; --j) {
            double s = c[j];
            for (int jj = j + 1; jj < k; ++jj) s -= A[(size_t)jj * m + j] * x[jj];
            x[j] = s / A[(size_t)j * m + j];
        }
    }
    if (resid) {
        double rr = 0.0;
        for (int i = 0; i < m; ++i) {
            double s = -b0[i];
            for (int j = 0; j < k; ++j) s += A0[(size_t)j * m + i] * x[j];
            rr += s * s;
        }
        *resid = sqrt(rr);
    }
    free(A); free(c); free(v);
    return deficient;
}

/* ---------------------------------------------------------------------- SPAI */

void orc_row_absmax_scale(int n, const int* rp, const double* av, double* d) {
    for (int j = 0; j < n; ++j) {
        double mx = 0.0;
        for (int p = rp[j]; p < rp[j + 1]; ++p) mx = fmax(mx, fabs(av[p]));
        d[j] = mx > 0.0 ? 1.0 / mx : 1.0;
    }
}

static int cmp_int(const void* a, const void* b) {
    int x = *(const int*)a, y = *(const int*)b;
    return (x > y) - (x < y);
}

int orc_spai(int n, const int* arp, const int* aci, const double* av,
             const int* prp, const int* pci, double spai_eps, double u_f,
             int col_begin, int col_end,
             double* mval, double* resid, int* conv, int* rankdef, double* kappa) {
    double* d = (double*)malloc(sizeof(double) * (size_t)n);
    orc_row_absmax_scale(n, arp, av, d);
    int nbad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : nbad)
    for (int k = col_begin; k < col_end; ++k) {
        /* J_k: pattern of column k of M' (row k of M), ascending */
        int nJ = prp[k + 1] - prp[k];
        const int* J = pci + prp[k];
        /* shadow I_k = union over j in J_k of the nonzero rows of column j of
           B = A^T D, i.e. of the columns of row j of A */
        int cand = 0;
        for (int q = 0; q < nJ; ++q) cand += arp[J[q] + 1] - arp[J[q]];
        int* I = (int*)malloc(sizeof(int) * (size_t)(cand > 0 ? cand : 1));
        int c = 0;
        for (int q = 0; q < nJ; ++q)
            for (int p = arp[J[q]]; p < arp[J[q] + 1]; ++p) I[c++] = aci[p];
        qsort(I, (size_t)c, sizeof(int), cmp_int);
        int nI = 0;
        for (int t = 0; t < c; ++t)
            if (nI == 0 || I[nI - 1] != I[t]) I[nI++] = I[t];
        /* Abar = B(I_k, J_k), column q holds row J[q] of A scaled by d_J[q] */
        double* Ab = (double*)calloc((size_t)nI * (size_t)(nJ > 0 ? nJ : 1), sizeof(double));
        double* e = (double*)calloc((size_t)(nI > 0 ? nI : 1), sizeof(double));
        double* mb = (double*)calloc((size_t)(nJ > 0 ? nJ : 1), sizeof(double));
        for (int q = 0; q < nJ; ++q) {
            int j = J[q];
            for (int p = arp[j]; p < arp[j + 1]; ++p) {
                int* hit = (int*)bsearch(&aci[p], I, (size_t)nI, sizeof(int), cmp_int);
                Ab[(size_t)q * nI + (hit - I)] = av[p] * d[j];
            }
        }
        for (int t = 0; t < nI; ++t) e[t] = (I[t] == k) ? 1.0 : 0.0;
        double fro = 0.0;
        for (size_t t = 0; t < (size_t)nI * (size_t)nJ; ++t) fro += Ab[t] * Ab[t];
        fro = sqrt(fro);
        double sres = 1.0;
        int rd = 0;
        double kap = 1.0;
        if (nJ > 0 && nI >= nJ) {
            rd = orc_householder_ls(nI, nJ, Ab, e, (double)nI * u_f * fro, mb, &sres);
            if (!rd && kappa) {
                /* kappa estimate ||R||_F ||R^-1||_F from a fresh QR of Abar */
                double* Q = (double*)malloc(sizeof(double) * (size_t)nI * nJ);
                memcpy(Q, Ab, sizeof(double) * (size_t)nI * nJ);
                double* R = (double*)calloc((size_t)nJ * nJ, sizeof(double));
                double* v = (double*)malloc(sizeof(double) * (size_t)nI);
                for (int j = 0; j < nJ; ++j) {
                    double sig = 0.0;
                    for (int i = j; i < nI; ++i) sig += Q[(size_t)j * nI + i] * Q[(size_t)j * nI + i];
                    sig = sqrt(sig);
                    double x0 = Q[(size_t)j * nI + j];
                    double sgn = x0 >= 0.0 ? 1.0 : -1.0;
                    for (int i = j; i < nI; ++i) v[i] = Q[(size_t)j * nI + i];
                    v[j] = x0 + sgn * sig;
                    double vtv = 0.0;
                    for (int i = j; i < nI; ++i) vtv += v[i] * v[i];
                    for (int jj = j; jj < nJ; ++jj) {
                        double dot = 0.0;
                        for (int i = j; i < nI; ++i) dot += v[i] * Q[(size_t)jj * nI + i];
                        for (int i = j; i < nI; ++i) Q[(size_t)jj * nI + i] -= 2.0 * dot / vtv * v[i];
                    }
                    for (int jj = j; jj < nJ; ++jj) R[(size_t)jj * nJ + j] = Q[(size_t)jj * nI + j];
                }
                double rf2 = 0.0, ri2 = 0.0;
                for (int t = 0; t < nJ * nJ; ++t) rf2 += R[t] * R[t];
                /* columns of R^-1 by back substitution */
                double* col = (double*)malloc(sizeof(double) * (size_t)nJ);
                for (int cc = 0; cc < nJ; ++cc) {
                    for (int j = nJ - 1; j >= 0; --j) {
                        double s = (j == cc) ? 1.0 : 0.0;
                        for (int jj = j + 1; jj < nJ; ++jj) s -= R[(size_t)jj * nJ + j] * col[jj];
                        col[j] = s / R[(size_t)j * nJ + j];
                        ri2 += col[j] * col[j];
                    }
                }
                kap = sqrt(rf2) * sqrt(ri2);
                free(col); free(Q); free(R); free(v);
            }
        } else if (nJ > 0) {
            rd = 1;
        }
        if (rd) {
            for (int q = 0; q < nJ; ++q) mb[q] = 0.0;
            sres = 1.0;
        }
        /* M = M'^T D: M[k, J[q]] = mbar[q] d_J[q] */
        for (int q = 0; q < nJ; ++q) mval[prp[k] + q] = mb[q] * d[J[q]];
        if (resid) resid[k] = sres;
        if (conv) conv[k] = (sres <= spai_eps);
        if (rankdef) rankdef[k] = rd;
        if (kappa) kappa[k] = kap;
        nbad += rd;
        free(I); free(Ab); free(e); free(mb);
    }
    free(d);
    return nbad;
}

/* ------------------------------------------------------- adaptive SPAI (f1) */

/* One pass of Alg 2.1's inner loop for column k of M' (SPAI on B = A^T D),
 * with the current pattern J (nJ indices, ascending):
 *   I      = shadow of J: the union of the columns of rows J of A (ascending);
 *   Abar   = B(I, J), ebar = e_k(I); mbar from Householder least squares;
 *   sbar   = Abar mbar - ebar (explicit, fp64), sres = ||sbar||_2;
 *   L      = I u {k}; Jt = (union over l in L of N_l) \ J, where N_l = {j :
 *            b_lj != 0} = the rows of A with an entry in column l (row l of
 *            A^T, given as trp/tci), ascending;
 *   rho_j  = sqrt(||sbar||^2 - (sbar^T B(I, j))^2 / ||B e_j||^2) for j in Jt,
 *            the residual norm after the best update along e_j alone;
 *   mean   = the arithmetic mean of rho over Jt;
 *   picks  = the up to beta indices of smallest rho (ties: smaller j) among
 *            those with rho_j <= mean.
 * The candidate part is skipped (ncand = npick = 0) when want_cand is 0.
 * cand/rho need room for every candidate (the caller sizes them by the
 * gathered count), picks for beta.  Returns the shadow size nI; *rd is the
 * rank flag (|R_jj| <= |I| u_f ||Abar||_F or |I| < |J|), in which case mbar = 0
 * and sres = 1. */
static int cmp_rho(const void* a, const void* b) {
    const double* x = (const double*)a;
    const double* y = (const double*)b;
    if (x[0] < y[0]) return -1;
    if (x[0] > y[0]) return 1;
    return (x[1] > y[1]) - (x[1] < y[1]);
}

static int shadow_of(const int* arp, const int* aci, const int* J, int nJ, int* I) {
    int c = 0;
    for (int q = 0; q < nJ; ++q)
        for (int p = arp[J[q]]; p < arp[J[q] + 1]; ++p) I[c++] = aci[p];
    qsort(I, (size_t)c, sizeof(int), cmp_int);
    int nI = 0;
    for (int t = 0; t < c; ++t)
        if (nI == 0 || I[nI - 1] != I[t]) I[nI++] = I[t];
    return nI;
}

int orc_spai_score(int n, const int* arp, const int* aci, const double* av, const int* trp,
                   const int* tci, const double* d, int k, const int* J, int nJ, double u_f,
                   int beta, int want_cand, double* mbar, double* sres, int* rd, int* cand,
                   double* rho, int* ncand, double* mean, int* picks, int* npick) {
    (void)n;
    int gathered = 0;
    for (int q = 0; q < nJ; ++q) gathered += arp[J[q] + 1] - arp[J[q]];
    int* I = (int*)malloc(sizeof(int) * (size_t)(gathered > 0 ? gathered : 1));
    const int nI = shadow_of(arp, aci, J, nJ, I);
    double* Ab = (double*)calloc((size_t)nI * (size_t)(nJ > 0 ? nJ : 1) + 1, sizeof(double));
    double* e = (double*)calloc((size_t)nI + 1, sizeof(double));
    double* sb = (double*)calloc((size_t)nI + 1, sizeof(double));
    for (int q = 0; q < nJ; ++q) {
        const int j = J[q];
        for (int p = arp[j]; p < arp[j + 1]; ++p) {
            const int* hit = (const int*)bsearch(&aci[p], I, (size_t)nI, sizeof(int), cmp_int);
            Ab[(size_t)q * nI + (size_t)(hit - I)] = av[p] * d[j];
        }
    }
    int pk = -1;
    for (int t = 0; t < nI; ++t)
        if (I[t] == k) { e[t] = 1.0; pk = t; }
    double fro = 0.0;
    for (size_t t = 0; t < (size_t)nI * (size_t)nJ; ++t) fro += Ab[t] * Ab[t];
    fro = sqrt(fro);
    double res = 1.0;
    *rd = 0;
    if (nJ == 0 || nI < nJ) {
        *rd = 1;
    } else {
        *rd = orc_householder_ls(nI, nJ, Ab, e, (double)nI * u_f * fro, mbar, &res);
    }
    if (*rd) {
        for (int q = 0; q < nJ; ++q) mbar[q] = 0.0;
        *sres = 1.0;
        *ncand = 0;
        *npick = 0;
        *mean = 0.0;
        free(I); free(Ab); free(e); free(sb);
        return nI;
    }
    /* sbar = Abar mbar - ebar, and its norm */
    double s2 = 0.0;
    for (int t = 0; t < nI; ++t) {
        double acc = -e[t];
        for (int q = 0; q < nJ; ++q) acc += Ab[(size_t)q * nI + t] * mbar[q];
        sb[t] = acc;
        s2 += acc * acc;
    }
    *sres = sqrt(s2);
    *ncand = 0;
    *npick = 0;
    *mean = 0.0;
    if (want_cand) {
        /* L = I u {k} */
        int nL = nI + (pk < 0 ? 1 : 0);
        int raw = 0;
        for (int t = 0; t < nL; ++t) {
            const int l = t < nI ? I[t] : k;
            raw += trp[l + 1] - trp[l];
        }
        int* C = (int*)malloc(sizeof(int) * (size_t)(raw > 0 ? raw : 1));
        int c = 0;
        for (int t = 0; t < nL; ++t) {
            const int l = t < nI ? I[t] : k;
            for (int p = trp[l]; p < trp[l + 1]; ++p) C[c++] = tci[p];
        }
        qsort(C, (size_t)c, sizeof(int), cmp_int);
        int nc = 0;
        for (int t = 0; t < c; ++t) {
            if (t > 0 && C[t] == C[t - 1]) continue;
            if (bsearch(&C[t], J, (size_t)nJ, sizeof(int), cmp_int)) continue;
            cand[nc++] = C[t];
        }
        double rsum = 0.0;
        for (int t = 0; t < nc; ++t) {
            const int j = cand[t];
            /* the residual of the univariate update m_k + mu e_j: the full
               residual is sbar on I (zero elsewhere), so sbar^T B e_j runs over
               the entries of column j of B (row j of A) that lie in I, and the
               denominator is the whole column's ||B e_j||^2 */
            double num = 0.0, den = 0.0;
            for (int p = arp[j]; p < arp[j + 1]; ++p) {
                const double bij = av[p] * d[j];
                den += bij * bij;
                const int* hit = (const int*)bsearch(&aci[p], I, (size_t)nI, sizeof(int), cmp_int);
                if (hit) num += sb[hit - I] * bij;
            }
            double r2 = s2;
            if (den > 0.0) r2 = s2 - num * num / den;
            rho[t] = sqrt(r2 > 0.0 ? r2 : 0.0);
            rsum += rho[t];
        }
        *ncand = nc;
        if (nc > 0) {
            *mean = rsum / nc;
            double* pr = (double*)malloc(sizeof(double) * 2 * (size_t)nc);
            for (int t = 0; t < nc; ++t) { pr[2 * t] = rho[t]; pr[2 * t + 1] = (double)cand[t]; }
            qsort(pr, (size_t)nc, 2 * sizeof(double), cmp_rho);
            int np = 0;
            for (int t = 0; t < nc && np < beta; ++t)
                if (pr[2 * t] <= *mean) picks[np++] = (int)pr[2 * t + 1];
            *npick = np;
            free(pr);
        }
        free(C);
    }
    free(I); free(Ab); free(e); free(sb);
    return nI;
}

int orc_spai_adaptive(int n, const int* arp, const int* aci, const double* av, const int* trp,
                      const int* tci, double spai_eps, double u_f, int alpha, int beta,
                      int imax_rows, int col_begin, int col_end, int cap, int* Jout, double* mout,
                      int* nJout, signed char* step_added, double* resid, int* conv, int* rankdef,
                      int* nsolves, int* capped) {
    double* d = (double*)malloc(sizeof(double) * (size_t)n);
    orc_row_absmax_scale(n, arp, av, d);
    int nbad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : nbad)
    for (int k = col_begin; k < col_end; ++k) {
        int* J = (int*)malloc(sizeof(int) * (size_t)cap);
        signed char* st = (signed char*)malloc((size_t)cap);
        double* mb = (double*)malloc(sizeof(double) * (size_t)cap);
        int* picks = (int*)malloc(sizeof(int) * (size_t)(beta > 0 ? beta : 1));
        int nJ = 1;
        J[0] = k;
        st[0] = 0;
        double sres = 1.0;
        int rd = 0, solves = 0, cp = 0;
        for (int step = 0; step <= alpha; ++step) {
            /* room for every candidate: at most sum over l in I u {k} of |N_l|,
               bounded by the entries of the rows of A^T over the gathered shadow */
            int gathered = 0;
            for (int q = 0; q < nJ; ++q) gathered += arp[J[q] + 1] - arp[J[q]];
            int* Itmp = (int*)malloc(sizeof(int) * (size_t)(gathered > 0 ? gathered : 1));
            const int nI0 = shadow_of(arp, aci, J, nJ, Itmp);
            int raw = trp[k + 1] - trp[k];
            for (int t = 0; t < nI0; ++t) raw += trp[Itmp[t] + 1] - trp[Itmp[t]];
            free(Itmp);
            int* cand = (int*)malloc(sizeof(int) * (size_t)(raw > 0 ? raw : 1));
            double* rho = (double*)malloc(sizeof(double) * (size_t)(raw > 0 ? raw : 1));
            int ncand = 0, npick = 0;
            double mean = 0.0;
            const int last = (step == alpha);
            orc_spai_score(n, arp, aci, av, trp, tci, d, k, J, nJ, u_f, beta, !last, mb, &sres, &rd,
                           cand, rho, &ncand, &mean, picks, &npick);
            ++solves;
            free(cand);
            free(rho);
            if (rd || sres <= spai_eps || last || npick == 0) break;
            /* J u picks, ascending; a pattern whose shadow would exceed imax_rows
               rows (or whose size would exceed cap) is not taken */
            int* Jn = (int*)malloc(sizeof(int) * (size_t)(nJ + npick));
            signed char* sn = (signed char*)malloc((size_t)(nJ + npick));
            int a = 0, b = 0, c = 0;
            int* pk2 = (int*)malloc(sizeof(int) * (size_t)npick);
            memcpy(pk2, picks, sizeof(int) * (size_t)npick);
            qsort(pk2, (size_t)npick, sizeof(int), cmp_int);
            while (a < nJ || b < npick) {
                if (b >= npick || (a < nJ && J[a] < pk2[b])) { Jn[c] = J[a]; sn[c++] = st[a++]; }
                else { Jn[c] = pk2[b++]; sn[c++] = (signed char)(step + 1); }
            }
            int g2 = 0;
            for (int q = 0; q < c; ++q) g2 += arp[Jn[q] + 1] - arp[Jn[q]];
            int* I2 = (int*)malloc(sizeof(int) * (size_t)(g2 > 0 ? g2 : 1));
            const int nI2 = shadow_of(arp, aci, Jn, c, I2);
            free(I2);
            free(pk2);
            if (c > cap || nI2 > imax_rows) {
                cp = 1;
                free(Jn); free(sn);
                break;
            }
            memcpy(J, Jn, sizeof(int) * (size_t)c);
            memcpy(st, sn, (size_t)c);
            nJ = c;
            free(Jn); free(sn);
        }
        for (int q = 0; q < nJ; ++q) {
            Jout[(size_t)k * cap + q] = J[q];
            mout[(size_t)k * cap + q] = rd ? 0.0 : mb[q] * d[J[q]];
            step_added[(size_t)k * cap + q] = st[q];
        }
        nJout[k] = nJ;
        resid[k] = rd ? 1.0 : sres;
        conv[k] = !rd && sres <= spai_eps;
        rankdef[k] = rd;
        nsolves[k] = solves;
        capped[k] = cp;
        nbad += rd;
        free(J); free(st); free(mb); free(picks);
    }
    free(d);
    return nbad;
}

/* ----------------------------------------------------------------- bucketing */

double orc_norm_inf(int n, const int* rp, const double* val) {
    double mx = 0.0;
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) s += fabs(val[p]);
        if (s > mx) mx = s;
    }
    return mx;
}

int orc_bucket_ids(int n, const int* rp, const double* val, double bucket_eps,
                   const int* fmts, int q, int8_t* id, int64_t* nnz_k, double* thr,
                   double* norm_out) {
    if (q < 1 || q > 8) return -1;
    for (int b = 1; b < q; ++b)
        if (!(orc_unit_roundoff(fmts[b]) > orc_unit_roundoff(fmts[b - 1]))) return -1;
    double nrm = orc_norm_inf(n, rp, val);
    double t[8];
    t[0] = INFINITY;
    for (int b = 1; b < q; ++b) t[b] = bucket_eps * nrm / orc_unit_roundoff(fmts[b]);
    for (int b = 0; b < q; ++b) { nnz_k[b] = 0; if (thr) thr[b] = t[b]; }
    for (int i = 0; i < n; ++i) {
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            double a = fabs(val[p]);
            int k = 0;
            if (q == 1 || a > t[1]) {
                k = 0;                         /* (eps ||A|| / u_2, inf) */
            } else if (a <= t[q - 1]) {
                k = q - 1;                     /* [0, eps ||A|| / u_q] */
            } else {
                for (int b = 1; b <= q - 2; ++b)   /* (eps ||A||/u_{k+1}, eps ||A||/u_k] */
                    if (a > t[b + 1] && a <= t[b]) k = b;
            }
            id[p] = (int8_t)k;
            nnz_k[k]++;
        }
    }
    if (norm_out) *norm_out = nrm;
    return 0;
}

/* Componentwise, x-dependent bucketing: the other strategy of Graillat et al.
 * that Section 2.3 mentions (and sets aside, because the buckets depend on the
 * vector x and must be redone for every product).  The paper does not state
 * it; this is the reading used here.  Row i: s_i = (|A||x|)_i, the fp64 sum in
 * ascending column order of the fp64 products |a_ij| |x_j|; thresholds
 * t_ik = eps s_i / u_k; element (i, j) goes to a bucket by the intervals of
 * eq. (nint) with |a_ij| replaced by |a_ij| |x_j| and ||A|| by s_i.  Bucket k
 * then holds products summing to at most p_ik eps s_i / u_k, so the bucketed
 * product (Alg 2.3 with these buckets) has componentwise backward error
 * max_i |yhat_i - y_i| / (|A||x|)_i within (q - 1) u_1 + c eps, c of
 * eq. (ccw) -- the normwise bound's form, row by row (pinned by exact
 * rationals in the tests). */
int orc_bucket_ids_cw(int n, const int* rp, const int* ci, const double* val, const double* x,
                      double bucket_eps, const int* fmts, int q, int8_t* id, int64_t* nnz_k, double* srow) {
    if (q < 1 || q > 8) return -1;
    for (int b = 1; b < q; ++b)
        if (!(orc_unit_roundoff(fmts[b]) > orc_unit_roundoff(fmts[b - 1]))) return -1;
    for (int b = 0; b < q; ++b) nnz_k[b] = 0;
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) s += fabs(val[p]) * fabs(x[ci[p]]);
        if (srow) srow[i] = s;
        double t[8];
        t[0] = INFINITY;
        for (int b = 1; b < q; ++b) t[b] = bucket_eps * s / orc_unit_roundoff(fmts[b]);
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            double a = fabs(val[p]) * fabs(x[ci[p]]);
            int k = 0;
            if (q == 1 || a > t[1]) {
                k = 0;
            } else if (a <= t[q - 1]) {
                k = q - 1;
            } else {
                for (int b = 1; b <= q - 2; ++b)
                    if (a > t[b + 1] && a <= t[b]) k = b;
            }
            id[p] = (int8_t)k;
            nnz_k[k]++;
        }
    }
    return 0;
}

double orc_storage_pct(const int64_t* nnz_k, const int* fmts, int q, int last_bits) {
    double num = 0.0, tot = 0.0;
    for (int b = 0; b < q; ++b) {
        int bits = orc_fmt_bits(fmts[b]);
        if (b == q - 1 && fmts[b] == ORC_DROP) bits = last_bits;
        num += (double)nnz_k[b] * bits;
        tot += (double)nnz_k[b];
    }
    if (tot == 0.0) return 0.0;
    return 100.0 * num / (tot * orc_fmt_bits(fmts[0]));
}

/* least power of two s = 2^e with maxabs <= fmax * 2^e */
static double pow2_scale(double maxabs, double fmax) {
    if (!(maxabs > 0.0)) return 1.0;
    int E;
    frexp(maxabs / fmax, &E);
    int e = E - 2;
    while (maxabs > ldexp(fmax, e)) ++e;
    while (e > -1074 && maxabs <= ldexp(fmax, e - 1)) --e;
    return ldexp(1.0, e);
}

int orc_bucket_store(int n, const int* rp, const int* ci, const double* val,
                     const int8_t* id, const int* fmts, int q,
                     double* stored, double* bucket_scale, double* col_scale) {
    double bmax[8] = {0};
    double* cmax = (double*)calloc((size_t)n, sizeof(double));
    for (int i = 0; i < n; ++i)
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            double a = fabs(val[p]);
            int b = id[p];
            if (a > bmax[b]) bmax[b] = a;
            if (fmts[b] == ORC_E4M3 && a > cmax[ci[p]]) cmax[ci[p]] = a;
        }
    for (int b = 0; b < q; ++b)
        bucket_scale[b] = fmts[b] == ORC_FP16 ? pow2_scale(bmax[b], orc_fmt_max(ORC_FP16)) : 1.0;
    for (int j = 0; j < n; ++j) col_scale[j] = pow2_scale(cmax[j], orc_fmt_max(ORC_E4M3));
    for (int i = 0; i < n; ++i)
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            int b = id[p];
            double m = val[p];
            switch (fmts[b]) {
            case ORC_FP64: stored[p] = m; break;
            case ORC_FP32:
            case ORC_BF16: stored[p] = orc_round(m, fmts[b]); break;
            case ORC_FP16: stored[p] = bucket_scale[b] * orc_round(m / bucket_scale[b], ORC_FP16); break;
            case ORC_E4M3: stored[p] = col_scale[ci[p]] * orc_round(m / col_scale[ci[p]], ORC_E4M3); break;
            default: stored[p] = 0.0; break;
            }
        }
    free(cmax);
    return 0;
}

void orc_bspmv(int n, const int* rp, const int* ci, const double* stored,
               const int8_t* id, const int* fmts, int q, const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double yi = 0.0;
        for (int b = 0; b < q; ++b) {
            if (fmts[b] == ORC_DROP) continue;
            int wide = fmts[b] == ORC_FP64;
            double acc = 0.0;
            for (int p = rp[i]; p < rp[i + 1]; ++p) {
                if (id[p] != b) continue;
                if (wide) {
                    acc = acc + stored[p] * x[ci[p]];
                } else {
                    double xt = orc_round(x[ci[p]], ORC_FP32);
                    double pr = orc_round(stored[p] * xt, ORC_FP32);
                    acc = orc_round(acc + pr, ORC_FP32);
                }
            }
            yi = yi + acc;
        }
        y[i] = yi;
    }
}

void orc_bspmv_literal(int n, const int* rp, const int* ci, const double* val,
                       const int8_t* id, const int* fmts, int q, const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double yi = 0.0;
        for (int b = 0; b < q; ++b) {
            int f = fmts[b];
            if (f == ORC_DROP) continue;
            double acc = 0.0;
            for (int p = rp[i]; p < rp[i + 1]; ++p) {
                if (id[p] != b) continue;
                double pr = rf(orc_round(val[p], f) * orc_round(x[ci[p]], f), f);
                acc = rf(acc + pr, f);
            }
            yi = rf(yi + acc, fmts[0]);
        }
        y[i] = yi;
    }
}

void orc_spmv_prec(int n, const int* rp, const int* ci, const double* val, int f,
                   const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; ++p)
            acc = rf(acc + rf(rf(val[p], f) * rf(x[ci[p]], f), f), f);
        y[i] = acc;
    }
}

/* --------------------------------------------------------------------- GMRES */

/* Dot product in u_g: every product and every sum rounded to u_g, the sum
 * taken pairwise (halves of the vector summed recursively, runs of at most 8
 * terms sequentially).  The paper fixes the precision, not the order; the
 * pairwise order keeps the error bound at gamma_(log2 n + 8) instead of the
 * sequential gamma_n (with n = 2^21 and u_g = 2^-24 the latter is 1/8). */
static double dot_g(int n, const double* a, const double* b, int ug) {
    if (n <= 8) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s = rf(s + rf(a[i] * b[i], ug), ug);
        return s;
    }
    const int h = n / 2;
    return rf(dot_g(h, a, b, ug) + dot_g(n - h, a + h, b + h, ug), ug);
}

/* Wall-clock seconds of each Arnoldi step of the next orc_gmres call, for the
 * CPU-baseline timing: a measurement aid that changes no result.  Set it right
 * before the call (one caller at a time); the call clears it. */
static double* g_step_seconds = NULL;
void orc_gmres_time_steps(double* out) { g_step_seconds = out; }

int orc_gmres(const orc_system_t* S, const double* r, int ug, int up, double tau, int kmax,
              double* d, int* iters, double* relres) {
    return orc_gmres_target(S, r, ug, up, tau, 0.0, kmax, d, iters, relres, NULL, NULL);
}

int orc_gmres_target(const orc_system_t* S, const double* r, int ug, int up, double tau, double target, int kmax,
                     double* d, int* iters, double* relres, double* beta_out, double* res_out) {
    double* step_seconds = g_step_seconds;
    g_step_seconds = NULL;
    int n = S->n;
    double* V = (double*)malloc(sizeof(double) * (size_t)n * (size_t)(kmax + 1));
    double* H = (double*)calloc((size_t)(kmax + 1) * (size_t)kmax, sizeof(double));
    double* cs = (double*)calloc((size_t)kmax + 1, sizeof(double));
    double* sn = (double*)calloc((size_t)kmax + 1, sizeof(double));
    double* g = (double*)calloc((size_t)kmax + 2, sizeof(double));
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    double* z = (double*)malloc(sizeof(double) * (size_t)n);
    double* y = (double*)calloc((size_t)kmax + 1, sizeof(double));

    /* s = M r (bucketed), stored in u_g */
    orc_bspmv(n, S->mrp, S->mci, S->mstored, S->mid, S->fmts, S->q, r, z);
    for (int i = 0; i < n; ++i) z[i] = rf(z[i], ug);
    double beta = rf(sqrt(dot_g(n, z, z, ug)), ug);
    int k = 0;
    double res = 0.0;
    if (beta > 0.0) {
        for (int i = 0; i < n; ++i) V[i] = rf(z[i] / beta, ug);
        g[0] = beta;
        res = beta;
        for (int j = 0; j < kmax; ++j) {
            const double t_step = step_seconds ? omp_get_wtime() : 0.0;
            double* vj = V + (size_t)j * n;
            /* w = A v_j in u_p (or by the bucketed SpMV on A's buckets, eq. nbe2), stored
             * in u_g;  z = M w (bucketed), stored in u_g */
            if (S->astored)
                orc_bspmv(n, S->arp, S->aci, S->astored, S->aid, S->fmts, S->q, vj, w);
            else
                orc_spmv_prec(n, S->arp, S->aci, S->av, up, vj, w);
            for (int i = 0; i < n; ++i) w[i] = rf(w[i], ug);
            orc_bspmv(n, S->mrp, S->mci, S->mstored, S->mid, S->fmts, S->q, w, z);
            for (int i = 0; i < n; ++i) z[i] = rf(z[i], ug);
            /* modified Gram-Schmidt */
            double* h = H + (size_t)j * (kmax + 1);
            for (int i = 0; i <= j; ++i) {
                const double* vi = V + (size_t)i * n;
                double hij = dot_g(n, vi, z, ug);
                h[i] = hij;
                for (int t = 0; t < n; ++t) z[t] = rf(z[t] - rf(hij * vi[t], ug), ug);
            }
            double hn = rf(sqrt(dot_g(n, z, z, ug)), ug);
            h[j + 1] = hn;
            /* Givens rotations in fp64 */
            for (int i = 0; i < j; ++i) {
                double t1 = cs[i] * h[i] + sn[i] * h[i + 1];
                double t2 = -sn[i] * h[i] + cs[i] * h[i + 1];
                h[i] = t1;
                h[i + 1] = t2;
            }
            double a = h[j], bb = h[j + 1];
            double rr = sqrt(a * a + bb * bb);
            if (rr == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
            else { cs[j] = a / rr; sn[j] = bb / rr; }
            h[j] = rr;
            h[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            res = fabs(g[j + 1]);
            k = j + 1;
            /* the tau test, or |g_{j+1}| <= target when the caller fixes the level */
            if (res <= (target > 0.0 ? target : tau * beta) || hn == 0.0) {
                if (step_seconds) step_seconds[j] = omp_get_wtime() - t_step;
                break;
            }
            double* vn = V + (size_t)(j + 1) * n;
            for (int t = 0; t < n; ++t) vn[t] = rf(z[t] / hn, ug);
            if (step_seconds) step_seconds[j] = omp_get_wtime() - t_step;
        }
        /* y = R^-1 g, back substitution in fp64 */
        for (int i = k - 1; i >= 0; --i) {
            double s = g[i];
            for (int jj = i + 1; jj < k; ++jj) s -= H[(size_t)jj * (kmax + 1) + i] * y[jj];
            y[i] = s / H[(size_t)i * (kmax + 1) + i];
        }
    }
    /* d = V y in u_g, stored in fp64 */
    for (int t = 0; t < n; ++t) {
        double acc = 0.0;
        for (int j = 0; j < k; ++j) acc = rf(acc + rf(V[(size_t)j * n + t] * rf(y[j], ug), ug), ug);
        d[t] = acc;
    }
    if (iters) *iters = k;
    if (relres) *relres = beta > 0.0 ? res / beta : 0.0;
    if (beta_out) *beta_out = beta;
    if (res_out) *res_out = res;
    free(V); free(H); free(cs); free(sn); free(g); free(w); free(z); free(y);
    return 0;
}

/* The correction equation of one refinement step, A d = r, solved with a
 * Krylov basis of at most kmem + 1 vectors: restarted GMRES cycles of kmem
 * steps on (M A) e = M r_c, r_0 = r, r_c = r - A d_c in u_r (ur_dd: Dot2)
 * rounded to u (format uw), d_{c+1} = d_c + e_c in fp64 (e_c stored in u).
 * Cycle 0 stops by the tau test (|g| <= tau ||M r||_2, beta_0 = that norm);
 * every later cycle stops when |g| <= tau beta_0, the same level; cycles end
 * when one stops before its kmem steps, meets the level, breaks down, or when
 * they have taken kmax steps in all (at most ceil(kmax / kmem) cycles).
 * Returns the steps taken; *cycles = cycles run. */
static int gmres_restarted(const orc_system_t* S, const double* r, int ug, int up, double tau, int kmax, int kmem,
                           int uw, int ur_dd, double* d, double* relres, int* cycles) {
    const int n = S->n;
    double* rc = (double*)malloc(sizeof(double) * (size_t)n);
    double* e = (double*)malloc(sizeof(double) * (size_t)n);
    for (int t = 0; t < n; ++t) d[t] = 0.0;
    int steps = 0, c = 0;
    double beta0 = 0.0, lvl = 0.0, res = 0.0;
    while (steps < kmax) {
        const double* rin = r;
        if (c > 0) {
            if (ur_dd) orc_residual_dd(n, S->arp, S->aci, S->av, d, r, rc);
            else orc_residual_fp64(n, S->arp, S->aci, S->av, d, r, rc);
            for (int t = 0; t < n; ++t) rc[t] = rf(rc[t], uw);
            rin = rc;
        }
        int k = 0;
        double beta = 0.0;
        orc_gmres_target(S, rin, ug, up, tau, c == 0 ? 0.0 : lvl, kmem, e, &k, NULL, &beta, &res);
        if (c == 0) {
            beta0 = beta;
            lvl = tau * beta0;
        }
        for (int t = 0; t < n; ++t) d[t] = d[t] + rf(e[t], uw);
        steps += k;
        ++c;
        if (k < kmem || res <= lvl || !(beta > 0.0)) break;
    }
    if (relres) *relres = beta0 > 0.0 ? res / beta0 : 0.0;
    if (cycles) *cycles = c;
    free(rc); free(e);
    return steps;
}

static double vnorm_inf(int n, const double* v) {
    double m = 0.0;
    for (int i = 0; i < n; ++i) m = fmax(m, fabs(v[i]));
    return m;
}

int orc_gmres_ir(const orc_system_t* S, const double* muf, const double* b,
                 int ug, int up, double tau, int kmax, int imax, double u_work,
                 int uw, int ur_dd, int uf,
                 int x0_given, double* x, int* its, double* nbe, double* dx, int* stop) {
    return orc_gmres_ir_m(S, muf, b, ug, up, tau, kmax, 0, imax, u_work, uw, ur_dd, uf, x0_given, x, its, nbe, dx,
                          stop, NULL);
}

int orc_gmres_ir_m(const orc_system_t* S, const double* muf, const double* b,
                   int ug, int up, double tau, int kmax, int kmem, int imax, double u_work,
                   int uw, int ur_dd, int uf,
                   int x0_given, double* x, int* its, double* nbe, double* dx, int* stop, int* cycles) {
    int n = S->n;
    double* r = (double*)malloc(sizeof(double) * (size_t)n);
    double* d = (double*)malloc(sizeof(double) * (size_t)n);
    /* x0 = M b with the unbucketed M (values muf) in u_f arithmetic, stored in fp64 */
    if (!x0_given) orc_spmv_prec(n, S->mrp, S->mci, muf, uf, b, x);
    /* x is held in the working precision u */
    for (int t = 0; t < n; ++t) x[t] = rf(x[t], uw);
    double anorm = orc_norm_inf(n, S->arp, S->av);
    double bnorm = vnorm_inf(n, b);
    double dprev = INFINITY;
    int steps = 0;
    *stop = 0;
    for (int i = 0; i < imax; ++i) {
        /* r = b - A x in u_r, stored in u */
        if (ur_dd)
            orc_residual_dd(n, S->arp, S->aci, S->av, x, b, r);
        else
            orc_residual_fp64(n, S->arp, S->aci, S->av, x, b, r);
        for (int t = 0; t < n; ++t) r[t] = rf(r[t], uw);
        double e = vnorm_inf(n, r) / (anorm * vnorm_inf(n, x) + bnorm);
        nbe[i] = e;
        if (e <= u_work) { *stop = 1; its[i] = 0; dx[i] = 0.0; break; }
        int k = 0;
        if (kmem > 0 && kmem < kmax) {
            k = gmres_restarted(S, r, ug, up, tau, kmax, kmem, uw, ur_dd, d, NULL, cycles ? cycles + i : NULL);
        } else {
            orc_gmres(S, r, ug, up, tau, kmax, d, &k, NULL);
            if (cycles) cycles[i] = 1;
        }
        its[i] = k;
        /* x = x + d in u, the correction first stored in u */
        for (int t = 0; t < n; ++t) {
            d[t] = rf(d[t], uw);
            x[t] = rf(x[t] + d[t], uw);
        }
        steps = i + 1;
        double dn = vnorm_inf(n, d), xn = vnorm_inf(n, x);
        dx[i] = xn > 0.0 ? dn / xn : dn;
        if (dn <= u_work * xn) { *stop = 2; break; }
        if (i > 0 && dn > 0.9 * dprev) { *stop = 3; break; }
        dprev = dn;
    }
    free(r); free(d);
    return steps;
}
