/*
 * bspai_oracle.h -- CPU oracle for BSPAI-GMRES-IR (Khan & Carson, arXiv 2307.03914).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, sequential restatement of
 * the paper's algorithms used to check the CUDA path.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product path never calls it.  It shares no code with the CUDA library.
 *
 * Arithmetic: fp64 unless a routine emulates a lower precision; emulation
 * computes each +, -, *, /, sqrt in fp64 and rounds once to the target format
 * (exact emulation for fp32/bf16/fp16/e4m3 by the double-rounding theorem,
 * since 53 >= 2t + 2).  Build with -ffp-contract=off.
 *
 * Conventions: CSR with int32 row pointers and columns sorted ascending per
 * row; all arrays are host memory owned by the caller.
 */
#ifndef BSPAI_ORACLE_H
#define BSPAI_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Number formats (Table 2, plus bf16 and OCP e4m3; "drop" is u = 1). */
enum { ORC_FP64 = 0, ORC_FP32 = 1, ORC_FP16 = 2, ORC_BF16 = 3, ORC_E4M3 = 4, ORC_DROP = 5 };

int    orc_fmt_bits(int fmt);           /* storage bits: 64/32/16/16/8/0 */
double orc_unit_roundoff(int fmt);      /* 2^-t: 2^-53, 2^-24, 2^-11, 2^-8, 2^-4, 1 */
double orc_fmt_max(int fmt);            /* largest finite value */
double orc_round(double x, int fmt);    /* round-to-nearest-even into fmt, with its range */
void   orc_round_array(const double* x, double* y, int64_t n, int fmt);

void orc_set_threads(int nthreads);
int  orc_get_threads(void);

/* Residual with u_r ~ u^2 (compensated Dot2), Alg 3.1 line "compute r_i = b - A x_i". */
void orc_residual_dd(int n, const int* rp, const int* ci, const double* av,
                     const double* x, const double* b, double* r);

/* Residual in plain fp64 (u_r = double): every product and difference rounded. */
void orc_residual_fp64(int n, const int* rp, const int* ci, const double* av,
                       const double* x, const double* b, double* r);

/* Dense Householder least squares min ||b - A x||_2, A m-by-k column-major (m >= k).
 * Returns 0, or 1 if a diagonal of R is <= rank_tol.  resid = ||A x - b||_2. */
int orc_householder_ls(int m, int k, const double* A, const double* b, double rank_tol,
                       double* x, double* resid);

/* Column scaling of Section 4: d_j = 1 / max_i |a_ji| (row j of A). */
void orc_row_absmax_scale(int n, const int* rp, const double* av, double* d);

/* Fixed-pattern SPAI (Alg 2.1 with alpha = 0) run on B = A^T D, returning
 * M = M'^T D in the structure of `pattern` (row k of M = column k of M').
 * Columns [col_begin, col_end) are computed.  u_f only sets the rank test
 * |R_jj| <= |I| u_f ||Abar||_F.  Outputs per column k: resid[k] = ||sbar_k||_2,
 * conv[k] = (resid <= spai_eps), rankdef[k], kappa[k] = ||R||_F ||R^-1||_F. */
int orc_spai(int n, const int* arp, const int* aci, const double* av,
             const int* prp, const int* pci, double spai_eps, double u_f,
             int col_begin, int col_end,
             double* mval, double* resid, int* conv, int* rankdef, double* kappa);

/* Adaptive SPAI (Alg 2.1 with alpha > 0; Grote and Huckle's pattern growth),
 * run on B = A^T D from the identity pattern, M = M'^T D.  trp/tci: the CSR
 * structure of A^T (row l lists the rows of A with an entry in column l).
 * Per column k in [col_begin, col_end): up to alpha + 1 least-squares solves;
 * after a solve the column stops when ||sbar||_2 <= spai_eps, after the last
 * solve, when no index qualifies, or when J u picks would have a shadow of
 * more than imax_rows rows or more than cap indices (capped[k] = 1).
 * Outputs (cap slots per column): Jout (ascending), mout = M[k, J] = mbar d_J,
 * step_added (0 for k, s for an index added after solve s), nJout, resid
 * (||sbar||_2), conv, rankdef, nsolves, capped.  Returns the number of
 * rank-deficient columns. */
int orc_spai_adaptive(int n, const int* arp, const int* aci, const double* av, const int* trp,
                      const int* tci, double spai_eps, double u_f, int alpha, int beta,
                      int imax_rows, int col_begin, int col_end, int cap, int* Jout, double* mout,
                      int* nJout, signed char* step_added, double* resid, int* conv, int* rankdef,
                      int* nsolves, int* capped);

/* One scoring pass of the adaptive SPAI for column k and pattern J (the step
 * that orc_spai_adaptive repeats): mbar, ||sbar||, the candidate indices with
 * their rho, the mean of rho and the picks.  d: the Section 4 scaling. */
int orc_spai_score(int n, const int* arp, const int* aci, const double* av, const int* trp,
                   const int* tci, const double* d, int k, const int* J, int nJ, double u_f,
                   int beta, int want_cand, double* mbar, double* sres, int* rd, int* cand,
                   double* rho, int* ncand, double* mean, int* picks, int* npick);


/* ||M||_inf = max_i sum_j |m_ij| (sequential, ascending column). */
double orc_norm_inf(int n, const int* rp, const double* val);

/* Bucketing, eq. (nint) / Alg 2.2: bucket ids 0..q-1 for every nonzero.
 * fmts[0..q-1] must have strictly increasing unit roundoff.  thr[b] =
 * bucket_eps ||M||_inf / u_b for b >= 1 (thr[0] = +inf).  Returns 0 or -1. */
int orc_bucket_ids(int n, const int* rp, const double* val, double bucket_eps,
                   const int* fmts, int q, int8_t* id, int64_t* nnz_k, double* thr,
                   double* norm_out);

/* Storage cost sum_k nnz_k bits_k / (nnz bits_0) in percent; the last bucket
 * is costed at last_bits when it is the drop format (0 or 8, see Tables 3/4). */
/* Componentwise (x-dependent) bucketing: s_i = (|A||x|)_i and the intervals of
 * eq. (nint) on |a_ij| |x_j| against eps s_i / u_k, per row.  srow may be NULL. */
int orc_bucket_ids_cw(int n, const int* rp, const int* ci, const double* val, const double* x,
                      double bucket_eps, const int* fmts, int q, int8_t* id, int64_t* nnz_k, double* srow);
double orc_storage_pct(const int64_t* nnz_k, const int* fmts, int q, int last_bits);

/* Stored values mtilde of each nonzero (scaled storage):
 *   fp64: m;  fp32, bf16: RN(m);  fp16: s_b RN16(m / s_b) with one power-of-two
 *   scale per bucket;  e4m3: s_j RNe4m3(m / s_j) with one power-of-two scale per
 *   column;  drop: 0.   s = 2^e with the least e such that max|m| <= fmt_max 2^e.
 * bucket_scale[q], col_scale[n] (1 where unused). */
int orc_bucket_store(int n, const int* rp, const int* ci, const double* val,
                     const int8_t* id, const int* fmts, int q,
                     double* stored, double* bucket_scale, double* col_scale);

/* Bucketed SpMV (Alg 2.3), decoupled form: each bucket's partial sum is
 * accumulated sequentially in ascending column order, in fp64 for an fp64
 * bucket and in fp32 (x rounded to fp32) for the narrower buckets; the
 * partial sums are added in fp64 in ascending bucket order. */
void orc_bspmv(int n, const int* rp, const int* ci, const double* stored,
               const int8_t* id, const int* fmts, int q, const double* x, double* y);

/* Paper-literal Alg 2.3: bucket k stored, and its partial sum computed, in
 * u_k with the format's own range (no scaling); sum over buckets in u_0. */
void orc_bspmv_literal(int n, const int* rp, const int* ci, const double* val,
                       const int8_t* id, const int* fmts, int q, const double* x, double* y);

/* Uniform-precision SpMV y = A x with values and x rounded to fmt and products
 * and sums in fmt (fp32 or fp64), sequential per row. */
void orc_spmv_prec(int n, const int* rp, const int* ci, const double* val, int fmt,
                   const double* x, double* y);

/* Left-preconditioned MGS-GMRES on (M A) d = M r (Alg 3.1, GMRES line).
 * Vector work in u_g (fp32/fp64), A v in u_p, M v bucketed (orc_bspmv);
 * Givens rotations and the triangular solve in fp64.  x0 = 0.
 * Stops when |g_{j+1}| <= tau ||M r||_2, on breakdown, or at kmax.
 * Outputs d (fp64), *iters, *relres = |g_k| / ||M r||_2.  Returns 0. */
typedef struct {
    int n;
    const int* arp; const int* aci; const double* av;          /* A */
    const int* mrp; const int* mci; const double* mstored;     /* bucketed M */
    const int8_t* mid; const int* fmts; int q;
    /* bucketed A (Section 3, eq. nbe2): stored values and bucket ids on A's
     * pattern, same formats as M; astored == NULL: A v in u_p */
    const double* astored; const int8_t* aid;
} orc_system_t;

/* Records the wall time of each Arnoldi step of the next orc_gmres call into
 * out[0 .. k-1] (timing aid only; no result changes). */
void orc_gmres_time_steps(double* out);
int orc_gmres(const orc_system_t* S, const double* r, int ug, int up, double tau, int kmax,
              double* d, int* iters, double* relres);
/* orc_gmres stopping at |g_{j+1}| <= target instead of the tau test when
 * target > 0; also returns beta = ||M r||_2 (in u_g) and the last |g|. */
int orc_gmres_target(const orc_system_t* S, const double* r, int ug, int up, double tau, double target, int kmax,
                     double* d, int* iters, double* relres, double* beta_out, double* res_out);

/* BSPAI-GMRES-IR driver (Alg 3.1 after the SPAI build).
 *   x0 = M b with the unbucketed M (values muf, arithmetic in u_f = format uf:
 *   ORC_FP32 or ORC_FP16) unless x0_given,
 *   rounded to the working precision u (format uw: ORC_FP64 or ORC_FP32);
 *   loop i < imax: r = b - A x in u_r (ur_dd = 1: Dot2, u_r ~ u^2; 0: plain
 *   fp64), rounded to u; nbe = ||r||_inf / (||A||_inf ||x||_inf + ||b||_inf);
 *   stop if nbe <= u_work; d = GMRES, rounded to u; x = fl_u(x + d); stop if
 *   ||d||_inf <= u_work ||x||_inf, or if ||d_i|| > 0.9 ||d_{i-1}||.
 * its[i] = GMRES iterations of step i; nbe[i], dx[i] histories; returns the
 * number of refinement steps taken.  *stop = 1 (nbe), 2 (dx), 3 (stagnation),
 * 0 (imax). */
int orc_gmres_ir(const orc_system_t* S, const double* muf, const double* b,
                 int ug, int up, double tau, int kmax, int imax, double u_work,
                 int uw, int ur_dd, int uf, int x0_given, double* x, int* its, double* nbe, double* dx, int* stop);
/* The same driver with the Krylov basis capped at kmem + 1 vectors (kmem > 0
 * and < kmax): each refinement step solves its correction equation by
 * restarted GMRES cycles of kmem steps (see gmres_restarted: later cycles
 * start from r - A d in u_r and stop at the first cycle's tau level), its[i]
 * counting the steps of all cycles and cycles[i] (may be NULL) the cycles. */
int orc_gmres_ir_m(const orc_system_t* S, const double* muf, const double* b,
                   int ug, int up, double tau, int kmax, int kmem, int imax, double u_work,
                   int uw, int ur_dd, int uf,
                   int x0_given, double* x, int* its, double* nbe, double* dx, int* stop, int* cycles);

#ifdef __cplusplus
}
#endif
#endif
