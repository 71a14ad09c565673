/*
 * bspai.h -- C ABI of the GB300 (sm_103a) BSPAI-GMRES-IR library, libbspai.so.
 *
 * Method: Khan & Carson, "Mixed Precision Iterative Refinement with Adaptive
 * Precision Sparse Approximate Inverse Preconditioning" (arXiv 2307.03914):
 *   - fixed-pattern sparse approximate inverse M (Section 2.2, eq. fronormmin,
 *     eq. redprob, Alg 2.1 with alpha = 0) built on A^T D with the column
 *     scaling of Section 4, then M = M'^T D (Alg 3.1, first line);
 *   - precision buckets of M by magnitude (eq. nint, Alg 2.2);
 *   - adaptive-precision SpMV (Alg 2.3);
 *   - left-preconditioned MGS-GMRES inside iterative refinement (Alg 3.1).
 *
 * Conventions for every call:
 *   - Pointers named as device pointers must be CUDA device memory on the
 *     current device; host pointers are ordinary host memory.  Caller-owned
 *     buffers stay owned by the caller; handles (bspai_A_h, bspai_M_h,
 *     bspai_BM_h) are owned by the library and released with bspai_free().
 *   - CSR inputs have int32 row pointers and int32 column indices sorted
 *     ascending within each row; nnz < 2^31.
 *   - All GPU work is enqueued on stream `s` (NULL = legacy default stream).
 *     Calls that fill an `info` struct synchronise `s` before returning;
 *     bspai_apply, bspai_apply_uf, bspai_residual and bspai_spmv_up do not.
 *   - Every call returns a bspai_status_t.  Nothing is thrown across the ABI.
 *     bspai_last_error() gives a per-thread message for the last failure.
 *   - Handles are not thread-safe: one handle, one thread at a time.
 */
#ifndef BSPAI_H
#define BSPAI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t (declared here so the header needs no CUDA headers). */
typedef struct CUstream_st* bspai_stream_t;

typedef enum {
    BSPAI_OK = 0,
    BSPAI_ERR_INVALID = 1,      /* bad argument (null pointer, size, unsorted precisions ...) */
    BSPAI_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    BSPAI_ERR_NOMEM = 3,        /* device allocation failed */
    BSPAI_NOT_CONVERGED = 4,    /* refinement hit i_max without meeting a stopping test */
    BSPAI_RANK_DEFICIENT = 5,   /* some SPAI least-squares block was rank deficient */
    BSPAI_NONFINITE = 6,        /* NaN or Inf in a residual or norm */
    BSPAI_TIMEOUT = 7,          /* a device-side grid barrier gave up after its time limit */
    BSPAI_ERR_UNSUPPORTED = 8   /* precision combination not built */
} bspai_status_t;

/* Number formats: Table 2 (half, single, double) plus bf16, OCP e4m3, "drop"
 * (u = 1, the element is removed, Section 4) and BSPAI_DD for u_r: a residual
 * as accurate as one carried in twice fp64 (compensated dot product Dot2). */
typedef enum {
    BSPAI_FP64 = 0,
    BSPAI_FP32 = 1,
    BSPAI_FP16 = 2,
    BSPAI_BF16 = 3,
    BSPAI_E4M3 = 4,
    BSPAI_DROP = 5,
    BSPAI_DD = 6
} bspai_prec_t;

/* A CSR matrix in device memory (caller-owned).  val may be NULL for a pattern. */
typedef struct {
    int32_t n;              /* order */
    int32_t nnz;            /* row_ptr[n] */
    const int32_t* row_ptr; /* device, n + 1 */
    const int32_t* col;     /* device, nnz, ascending within each row */
    const double* val;      /* device, nnz (fp64), or NULL */
} bspai_csr_t;

typedef struct bspai_matrix* bspai_A_h;   /* A prepared for the GPU kernels */
typedef struct bspai_spai* bspai_M_h;     /* M = SPAI(A) held in u_f (fp32 or fp16) */
typedef struct bspai_bucketed* bspai_BM_h;/* M split into precision buckets */

typedef struct {
    int32_t n;
    int32_t max_cols;          /* largest |J_k| */
    int32_t max_rows;          /* largest |I_k| (shadow size) */
    int32_t n_converged;       /* columns with ||sbar_k||_2 <= spai_eps (Alg 2.1 test) */
    int32_t n_rank_deficient;  /* columns whose block failed |R_jj| > |I| u_f ||Abar||_F */
    int64_t nnz;               /* nnz(M) (= nnz(pattern) for the fixed pattern) */
    double max_resid;          /* max_k ||sbar_k||_2 */
    int32_t n_capped;          /* adaptive build: columns whose growth stopped at imax_rows */
    int32_t n_second_tier;     /* adaptive build: columns rerun with the full per-column bounds */
    int64_t total_solves;      /* least-squares solves over all columns (n for the fixed pattern) */
} bspai_build_info_t;

typedef struct {
    int32_t q;                 /* number of buckets */
    int32_t precs[8];          /* bspai_prec_t of each bucket, increasing unit roundoff */
    int64_t nnz_k[8];          /* nonzeros per bucket (dropped ones counted in their bucket) */
    int64_t slots_k[8];        /* stored slots per bucket including padding */
    double thresholds[8];      /* thresholds[k] = eps ||M||_inf / u_k, k >= 1; [0] = +inf */
    double norm_inf;           /* ||M||_inf */
    double storage_pct;        /* sum_k nnz_k bits_k / (nnz bits_1), drop costed at 0 bits */
    double storage_pct_last8;  /* same with a dropped last bucket costed at 8 bits */
    int64_t bytes;             /* device bytes of the bucketed M (values, indices, scales) */
} bspai_bucket_info_t;

typedef struct {
    double tau;            /* GMRES tolerance: stop when |g_{j+1}| <= tau ||M r||_2 (Alg 3.1) */
    int32_t kmax;          /* max GMRES iterations per refinement step (no restart unless
                              basis_bytes_max asks); 0 = min(n, 1000) */
    int32_t i_max;         /* max refinement steps; 0 = 10 */
    int32_t x0_given;      /* 1: x holds the initial iterate; 0: x0 = M b in u_f (Alg 3.1) */
    int32_t max_blocks;    /* cap on the blocks (one per SM) of the cooperative GMRES kernels;
                              0 = every SM.  Several solves on different streams, each capped,
                              share the GPU concurrently (e.g. one solve per right-hand side). */
    double u_stop;         /* stop when nbe <= u_stop or ||d||_inf <= u_stop ||x||_inf; 0 = 2^-53 */
    double stagnation;     /* stop when ||d_i|| > stagnation ||d_{i-1}||; 0 = 0.9 */
    double barrier_timeout_s; /* device grid-barrier time limit in seconds; 0 = 2.0 */
    int64_t basis_bytes_max;  /* gmres_ir_solve*: cap on the device bytes of the Krylov basis
                                 ((m + 1) vectors of n in u_g, n rounded up to 64); 0 = none.
                                 When the kmax + 1 vectors exceed it, or their allocation fails
                                 for lack of device memory (m halved until it fits, m >= 8),
                                 each refinement step solves its correction equation by
                                 restarted GMRES cycles of m steps: cycle c > 0 starts from
                                 r - A d (u_r, stored in u), stops at the first cycle's level
                                 |g| <= tau ||M r||_2, and the cycles end when one stops early,
                                 meets that level, or they have taken kmax steps (at most
                                 ceil(kmax / m) cycles); d sums the cycles' corrections (each
                                 stored in u) in fp64.  The basis is rebuilt by each cycle
                                 instead of being stored whole.  A cap below two vectors:
                                 BSPAI_ERR_INVALID. */
} bspai_opts_t;

typedef struct {
    int32_t status;            /* bspai_status_t of the solve */
    int32_t ir_steps;          /* refinement steps that ran GMRES */
    int32_t stop_reason;       /* 1 nbe <= u, 2 ||d|| <= u ||x||, 3 stagnation, 0 i_max */
    int32_t total_iters;       /* sum of GMRES iterations */
    int32_t gmres_iters[32];   /* GMRES iterations of each refinement step */
    double nbe[33];            /* ||r||_inf / (||A||_inf ||x||_inf + ||b||_inf) at each residual */
    double dx[32];             /* ||d_i||_inf / ||x_{i+1}||_inf */
    double relres[32];         /* |g_k| / ||M r||_2 at the end of each GMRES */
    int32_t kmem;              /* steps per GMRES cycle the Krylov basis held (kmax unless capped) */
    int32_t gmres_cycles[32];  /* GMRES cycles of each refinement step (1 unless capped) */
} bspai_solve_info_t;

/* Kernel-class timing, recorded with CUDA events on the launching stream. */
enum {
    BSPAI_K_SPAI = 0, BSPAI_K_BUCKET = 1, BSPAI_K_SPMV_A = 2, BSPAI_K_BSPMV = 3,
    BSPAI_K_MGS = 4, BSPAI_K_RESIDUAL = 5, BSPAI_K_UPDATE = 6, BSPAI_K_OTHER = 7,
    BSPAI_K_COUNT = 8
};
typedef struct {
    double ms[BSPAI_K_COUNT];        /* summed event time per class */
    int64_t launches[BSPAI_K_COUNT]; /* kernel launches per class */
} bspai_profile_t;

/* ------------------------------------------------------------------ basics */
const char* bspai_last_error(void);       /* per-thread message; never NULL */
int bspai_version(void);                  /* 10000 * major + 100 * minor + patch */
/* Kernel launches this library has issued since it was loaded (all threads). */
long long bspai_launch_count(void);
/* Failure-detection self-test of the bounded grid barrier that the cooperative
 * GMRES kernels use (no counterpart in the paper).  Launches `blocks` CTAs
 * (1..1024, all co-resident: a cooperative launch) that meet once at that
 * barrier.  hold = 0: an ordinary barrier, returns BSPAI_OK.  hold != 0: the
 * arrival counter starts past the value at which the last arrival releases
 * the barrier, so no arrival releases it; every CTA gives up after
 * `timeout_s` seconds (0 < timeout_s <= 10) and the call returns
 * BSPAI_TIMEOUT.  No memory fault, trap or unbounded wait is involved and the
 * CUDA context stays usable.  Synchronises stream s.  *waited_ms, if not
 * NULL, receives the kernel's duration (CUDA events). */
int bspai_barrier_selftest(int blocks, int hold, double timeout_s, bspai_stream_t s, float* waited_ms);
void bspai_opts_default(bspai_opts_t* opts);
/* Measured issue rate of the SM's plain (non-tensor) fused multiply-add in
 * prec (BSPAI_FP32 or BSPAI_FP64; otherwise BSPAI_ERR_UNSUPPORTED): a
 * measurement aid with no counterpart in the paper, the denominator of the
 * ALU rooflines of the SPAI build (fp32) and the Dot2 residual (fp64).  Runs
 * eight 256-thread blocks per SM, every thread eight independent chains of
 * 32 x iters dependent FMAs (8 <= iters <= 2^24, else BSPAI_ERR_INVALID),
 * after one shorter warm-up launch, timed with CUDA events on stream s
 * (synchronised).  *fma_per_s: lane FMAs per second over the whole GPU
 * (flop/s = 2 x that); *ms (may be NULL): the timed launch's duration.
 * Allocates and frees a small device buffer. */
int bspai_probe_fma(bspai_prec_t prec, int32_t iters, bspai_stream_t s, double* fma_per_s, float* ms);

/* Releases any handle returned by this library (NULL is a no-op).  Enqueues
 * the frees on the stream the handle was created on. */
int bspai_free(void* handle);
/* Enables (1) or disables (0) per-kernel-class event timing for later calls. */
int bspai_profile_enable(int on);
/* Synchronises the recorded events and returns the totals; reset = 1 clears them. */
int bspai_profile_read(bspai_profile_t* out, int reset);

/* ------------------------------------------------------------------ componentwise study */
/* The componentwise, x-dependent bucketed product y = M x: Section 2.3 notes
 * that Graillat et al. also bucket by the products, for a componentwise
 * backward-error bound, and sets that aside because the buckets depend on x.
 * The paper does not print the rule; here, per row i, s_i = (|M||x|)_i (fp64,
 * ascending columns) and entry (i, j) goes to bucket k by the intervals of
 * eq. (nint) applied to fl64(|m_ij| |x_j|) against t_k = eps s_i / u_k.  The
 * product is then Alg 2.3 on those buckets, decoupled as bspai_apply (fp64
 * bucket in fp64, fp32 / bf16 buckets in fp32 with x rounded to fp32, partial
 * sums added in fp64 in bucket order).  Both steps run in one launch per
 * product, reading M in u_f (no stored buckets).  precs: q <= 4 of BSPAI_FP64,
 * BSPAI_FP32, BSPAI_BF16, BSPAI_DROP with increasing unit roundoff (fp16 and
 * e4m3 need a scale fitted to each bucket: BSPAI_ERR_UNSUPPORTED).  x, y:
 * device, n entries, FP64 or FP32.  ids (device int8, nnz(M), CSR order) and
 * nnz_k (host, q entries; the call then synchronises s) may be NULL. */
int bspai_apply_cw(bspai_M_h M, double bucket_eps, const int32_t* precs, int32_t q, const void* x,
                   bspai_prec_t x_prec, void* y, bspai_prec_t y_prec, int8_t* ids, int64_t* nnz_k,
                   bspai_stream_t s);

/* ------------------------------------------------------------------ A */
/* Prepares A (n x n, values required) for the kernels: sliced-ELL copies of
 * its structure with fp64 values (residual, u_r) and fp32 values (u_p).
 * A's buffers may be freed after the call's stream work completes. */
int bspai_matrix_create(const bspai_csr_t* A, bspai_stream_t s, bspai_A_h* out);

/* r = b - A x computed with u_r ~ u^2 (Dot2: TwoProduct by FMA, TwoSum; the
 * paper uses quad), stored in
 * fp64 (Alg 3.1, residual line).  x, b, r: device fp64 vectors of length n. */
int bspai_residual(bspai_A_h A, const double* x, const double* b, double* r, bspai_stream_t s);

/* r = b - A x computed in u_r and stored in the working precision u (Alg 3.1
 * residual line; Section 4's (single, single, double) setting has u_r = FP64,
 * u = FP32).  u_r: BSPAI_DD (as bspai_residual) or BSPAI_FP64 (every product
 * and difference rounded to fp64, ascending column order); u: BSPAI_FP64 or
 * BSPAI_FP32 (r rounded to fp32, held in the fp64 buffer).  x, b, r: device
 * fp64, length n.  Other precisions: BSPAI_ERR_UNSUPPORTED. */
int bspai_residual_prec(bspai_A_h A, const double* x, const double* b, bspai_prec_t u_r, bspai_prec_t u, double* r,
                        bspai_stream_t s);

/* w = A v with A rounded to u_p = fp32 and fp32 products and sums (Alg 3.1,
 * GMRES line: "A computed in precision u_p").  v, w: device fp32, length n. */
int bspai_spmv_up(bspai_A_h A, const float* v, float* w, bspai_stream_t s);

/* ------------------------------------------------------------------ SPAI */
/* Adaptive SPAI (Alg 2.1 with alpha > 0, Grote and Huckle's pattern growth)
 * run on B = A^T D from the identity pattern (Section 4), in u_f (BSPAI_FP32,
 * or BSPAI_FP16 with every operation in IEEE half as in bspai_build; the
 * candidate sums sbar^T B(I, j) are the u_f products added exactly, then
 * rounded once to u_f; other u_f: BSPAI_ERR_UNSUPPORTED), giving M = M'^T D.  Per column k, at most alpha + 1 passes of: shadow I_k,
 * least squares on B(I_k, J_k) by Householder QR, sbar; stop when ||sbar||_2
 * <= spai_eps or after the last pass; otherwise score every j in (union over
 * l in I_k u {k} of the nonzero columns of row l of B) \ J_k by
 * rho_j = (||sbar||^2 - (sbar^T B(I_k, j))^2 / ||B e_j||^2)^(1/2) and add
 * the up to beta of smallest rho_j (ties: smaller j) among those with rho_j
 * <= the mean rho.  A pass whose new pattern would have a shadow of more than
 * imax_rows rows is not taken (the column keeps its solution; counted in
 * info->n_capped).  imax_rows must be >= the longest row of A; the shared
 * memory of one column grows with 1 + alpha beta and imax_rows, and a
 * configuration that does not fit returns BSPAI_ERR_UNSUPPORTED.  0 <= alpha
 * <= 16, 0 <= beta <= 32.  A: device CSR (fp64 values).  The returned M works
 * wherever a fixed-pattern M does.  Returns BSPAI_RANK_DEFICIENT (M still
 * created) if any block failed the rank test, BSPAI_NONFINITE (M created) if
 * an entry of M overflowed the range of u_f. */
int bspai_build_adaptive(const bspai_csr_t* A, double spai_eps, int32_t alpha, int32_t beta, int32_t imax_rows,
                         bspai_prec_t u_f, bspai_stream_t s, bspai_M_h* M_out, bspai_build_info_t* info);

/* For an M from bspai_build_adaptive: per entry in CSR order, the pass that
 * added it (0 for the diagonal start, s for an index chosen after pass s;
 * int8, nnz(M)), and per column solves | converged << 8 | rank deficient << 9
 * | capped << 10 (int32, n).  Device buffers; either may be NULL.  Other
 * handles: BSPAI_ERR_UNSUPPORTED. */
int bspai_M_adaptive_export(bspai_M_h M, int8_t* step_added, int32_t* col_info, bspai_stream_t s);

/* Fixed-pattern SPAI (Alg 2.1 with alpha = 0; eq. redprob) run on B = A^T D,
 * D = diag(1 / max_i |a_ji|) (Section 4), in u_f, giving the left
 * preconditioner M = M'^T D (Alg 3.1, first line).  Row k of M has the
 * structure of row k of `pattern` (pattern->val is ignored).  For each k the
 * shadow I_k, the block Abar = B(I_k, J_k), its Householder QR, mbar =
 * R^-1 Q^T ebar and ||sbar_k||_2 are computed on the GPU, one warp per column.
 * u_f = BSPAI_FP32, or BSPAI_FP16 for the (half, single, double) setting of
 * Section 4: every operation of the solve is then an IEEE half operation (the
 * half format's own range; Section 4's scaling keeps B's entries in [-1, 1])
 * and M's entries are half values.  Other u_f: BSPAI_ERR_UNSUPPORTED.
 * Returns BSPAI_RANK_DEFICIENT (with M still created, those columns zero) if
 * any block failed the rank test, BSPAI_NONFINITE (M created) if an entry of
 * M = M'^T D overflowed the range of u_f. */
int bspai_build(const bspai_csr_t* A, const bspai_csr_t* pattern, double spai_eps,
                bspai_prec_t u_f, bspai_stream_t s, bspai_M_h* M_out, bspai_build_info_t* info);

/* Copies M out in CSR order (structure of the pattern): row_ptr (n+1), col
 * (nnz), val (nnz, fp32 holding the u_f values) and resid (n, ||sbar_k||_2 per
 * column of M' = row of M).  All device buffers; any may be NULL. */
int bspai_M_export(bspai_M_h M, int32_t* row_ptr, int32_t* col, float* val, float* resid,
                   bspai_stream_t s);

/* Creates an M handle from a sparse approximate inverse computed elsewhere:
 * Mcsr holds M (device CSR, fp64 values, rounded once to u_f: BSPAI_FP32 or
 * BSPAI_FP16, else BSPAI_ERR_UNSUPPORTED).  The handle behaves like one from
 * bspai_build (bucketing, x0 = M b in u_f), with zero column residuals. */
int bspai_M_create(const bspai_csr_t* Mcsr, bspai_prec_t u_f, bspai_stream_t s, bspai_M_h* M_out);

/* y = M x with the unbucketed M in its u_f (x rounded once to u_f, every
 * product and sum in u_f, columns in ascending order), y stored in fp64:
 * x0 = M b of Alg 3.1.  Device vectors. */
int bspai_apply_uf(bspai_M_h M, const double* x, double* y, bspai_stream_t s);

/* ------------------------------------------------------------------ buckets */
/* Splits M into q <= 8 precision buckets (eq. nint, Alg 2.2) with
 * ||M|| = ||M||_inf computed in fp64 (row sums in ascending column order).
 * precs[0..q-1] must have strictly increasing unit roundoff (fp64 < fp32 <
 * fp16 < bf16 < e4m3 < drop).  Storage: fp64/fp32/bf16 buckets hold RN(m);
 * an fp16 bucket holds RN16(m / s) with one power-of-two scale s per bucket;
 * an e4m3 bucket holds RNe4m3(m / s_j) with a power-of-two fp32 scale per
 * column (s = least 2^e with max|m| <= fmt_max 2^e); drop removes entries.
 * At most one e4m3 bucket.  Each bucket is a sliced ELL structure of 32-row
 * slices whose rows keep their slots in groups of four consecutive elements
 * (one vector load per row and group in bspai_apply), with column indices held
 * as 16-bit differences to the row when every |c - r| <= 32767, else int32.
 * BM keeps its own copy of everything it needs, so M may be freed afterwards. */
int bspai_bucket(bspai_M_h M, double bucket_eps, const int32_t* precs, int32_t q,
                 bspai_stream_t s, bspai_BM_h* out, bspai_bucket_info_t* info);

/* Bucketing of a batch of nsys independent systems stacked block-diagonally in
 * M (all systems built by one bspai_build call on the block-diagonal A and
 * pattern): system s owns rows row_off[s] .. row_off[s+1]-1 (device int32,
 * nsys + 1 entries, multiples of 32, row_off[0] = 0, row_off[nsys] = n; rows
 * that pad a system to a multiple of 32 have no entries).  Each system is
 * bucketed exactly as bspai_bucket would bucket it alone: its own ||M_s||_inf,
 * thresholds and fp16 scale (eq. nint per system).  info: bucket counts over
 * the whole batch, norm_inf = max_s ||M_s||_inf, thresholds of system 0. */
int bspai_bucket_batched(bspai_M_h M, const int32_t* row_off, int32_t nsys, double bucket_eps,
                         const int32_t* precs, int32_t q, bspai_stream_t s, bspai_BM_h* out,
                         bspai_bucket_info_t* info);

/* Buckets of A itself (Section 3, eq. nbe2: the adaptive-precision SpMV also
 * applied to A inside GMRES, with the same precision list and bucket_eps as
 * M): ||A||_inf from A's fp64 values, t_k = bucket_eps ||A||_inf / u_k, every
 * entry to its bucket by eq. (nint), stored in the bucket's format with one
 * rounding from fp64 (fp16 / e4m3 scaled as for M).  A: from
 * bspai_matrix_create (not a transposed A: BSPAI_ERR_UNSUPPORTED).  The result
 * is used by gmres_ir_solve_hb / bspai_gmres_b, and by bspai_apply (y = A x)
 * and bspai_bucket_export like a bucketed M. */
int bspai_bucket_A(bspai_A_h A, double bucket_eps, const int32_t* precs, int32_t q, bspai_stream_t s,
                   bspai_BM_h* out, bspai_bucket_info_t* info);

/* Per nonzero of M in CSR order: bucket id (0-based) and the stored value the
 * product uses (scale applied), as fp64.  Device buffers of length nnz(M);
 * either may be NULL. */
int bspai_bucket_export(bspai_BM_h BM, int8_t* ids, double* stored, bspai_stream_t s);

/* Which kernel form the sparse products (bspai_apply, A v and M w inside the
 * solvers) use.  All forms compute the same operations in the same order and
 * give identical bits.  BSPAI_SPMV_AUTO (default): kernels with the storage
 * format of every bucket fixed at compile time for the mixes the solvers meet
 * (one fp32 / fp64 / fp16 bucket, or fp16 + e4m3, fp32 + fp16, fp64 + fp32),
 * else the generic register form.  BSPAI_SPMV_REGISTERS: always the generic
 * register form.  BSPAI_SPMV_STAGED: the form whose matrix stream is staged
 * into shared memory by bulk copies (TMA) wherever it applies (large
 * matrices, at most 4 stored buckets), else the generic register form.
 * Process-wide; affects launches issued after the call.  No counterpart in
 * the paper. */
enum { BSPAI_SPMV_AUTO = 0, BSPAI_SPMV_REGISTERS = 1, BSPAI_SPMV_STAGED = 2 };
int bspai_set_spmv_form(int form);

/* y = M x by the adaptive-precision SpMV (Alg 2.3): per row and bucket a
 * partial sum accumulated in ascending column order, in fp64 for an fp64
 * bucket and in fp32 (x rounded to fp32) for narrower buckets (storage in
 * u_k, computation decoupled as in Section 5); partial sums added in fp64 in
 * bucket order; the result rounded to y_prec.  x_prec, y_prec in {FP64, FP32}. */
int bspai_apply(bspai_BM_h BM, const void* x, bspai_prec_t x_prec, void* y, bspai_prec_t y_prec,
                bspai_stream_t s);

/* ------------------------------------------------------------------ solves */
/* One left-preconditioned MGS-GMRES solve of (M A) d = M r (Alg 3.1, GMRES
 * line): vectors in u_g (FP32 or FP64), A v in u_p (FP32 or FP64), M v
 * bucketed (Alg 2.3), Givens rotations and the triangular solve in fp64;
 * x0 = 0, no restart, stop when |g_{j+1}| <= opts->tau ||M r||_2 or at kmax.
 * r and d are device fp64 vectors.  info->gmres_iters[0], relres[0] are set. */
int bspai_gmres(bspai_A_h A, bspai_BM_h BM, const double* r, bspai_prec_t u_g, bspai_prec_t u_p,
                const bspai_opts_t* opts, double* d, bspai_stream_t s, bspai_solve_info_t* info);

/* Which kernel runs the modified Gram-Schmidt step of the GMRES solves
 * (Alg 3.1, GMRES line; MGS as analysed in Section 3) for an order n, u_g in
 * {FP32, FP64}, and a cap max_blocks on the cooperative grid (0: every SM),
 * as bspai_gmres, gmres_ir_solve and their variants would pick it on the
 * current device.  kernel: 0 = k_mgs (basis and new vector streamed from
 * memory), 1 = k_mgs_res (the new vector held on chip; per_thread rows per
 * thread), 2 = k_mgs_res2 (fp32, the new vector in registers; per_thread
 * pairs of adjacent rows per thread); block_threads and blocks give the
 * launch; poll_bulk = 1 when the on-chip kernel's warp 0 reads the grid
 * reductions' slots by bulk copies into shared memory instead of by loads
 * (at least 16 KB of each basis vector per block and at least 64 blocks),
 * 0 otherwise.  A query only: nothing is launched or allocated.  n < 1:
 * BSPAI_ERR_INVALID; another u_g: BSPAI_ERR_UNSUPPORTED. */
typedef struct {
    int32_t kernel;
    int32_t per_thread;
    int32_t block_threads;
    int32_t blocks;
    int32_t poll_bulk;
} bspai_gmres_plan_t;
int bspai_gmres_plan(int32_t n, bspai_prec_t u_g, int32_t max_blocks, bspai_gmres_plan_t* out);

/* bspai_gmres with A v by the adaptive-precision SpMV on A's buckets
 * (bspai_bucket_A) instead of A in u_p (eq. nbe2); products accumulated as in
 * bspai_apply, results rounded to u_g.  A_bucketed must hold A's n rows (a
 * missing handle, another handle kind or another size: BSPAI_ERR_INVALID);
 * the other arguments and the returns are those of bspai_gmres. */
int bspai_gmres_b(bspai_A_h A, bspai_BM_h A_bucketed, bspai_BM_h BM, const double* r, bspai_prec_t u_g,
                  const bspai_opts_t* opts, double* d, bspai_stream_t s, bspai_solve_info_t* info);

/* The same GMRES solve as bspai_gmres, for callers that cannot allocate
 * device memory at the time of the call -- for example a host program that
 * has handed the GPU's memory to its own pool allocator up front, or one that
 * must not call cudaMalloc/cudaFree (which can synchronise the device) once
 * it is running.  The paper has no counterpart to this entry point; it only
 * changes where the workspace lives.
 *   - Workspace: one fixed 64 MiB block of device memory that belongs to the
 *     library image (every GPU that loads the library holds it until the
 *     process exits).  The call needs n_pad * (kmax + 1) values in u_g
 *     (n_pad = n rounded up to 64) plus about 8 (kmax + 1)^2 bytes; larger
 *     problems are rejected with BSPAI_ERR_INVALID and a message giving the
 *     bytes needed, and nothing is launched.
 *   - Nothing is allocated: no cudaMalloc, cudaFree or stream-ordered pool
 *     allocation, and no pinned host buffer.  (Leave kernel-class timing,
 *     bspai_profile_enable, off: it creates CUDA events.)
 *   - The first call on a device looks up the device address of the block
 *     with that device current; make that first call before any stream
 *     capture begins.  The address is kept per device together with the id
 *     of the CUDA context it was found in: after a device reset (a new
 *     context, in which the library's image may sit elsewhere) the next call
 *     looks it up again, so make that call before any capture as well.
 *   - Every call uses the same block, which keeps the previous call's
 *     contents; each call clears the parts that must start at zero.  Two calls
 *     whose GPU work overlaps (for example on two streams of one device) race
 *     on the block and give undefined results: run them one after another.
 * A, BM, r, d, opts and info as for bspai_gmres. */
int bspai_gmres_noalloc(bspai_A_h A, bspai_BM_h BM, const double* r, bspai_prec_t u_g, bspai_prec_t u_p,
                        const bspai_opts_t* opts, double* d, bspai_stream_t s, bspai_solve_info_t* info);

/* BSPAI-GMRES-IR (Alg 3.1 after the SPAI build): x0 = M b in u_f (unless
 * opts->x0_given), then up to i_max steps of r = b - A x in u_r, GMRES on
 * (M A) d = M r with tolerance tol, x = x + d in u.  Supported: u in {FP64,
 * FP32}, u_r in {DD, FP64}, u_g and u_p in {FP32, FP64}.  With u = FP32 (the
 * (single, single, double) setting of Section 4) x, r and d are held in fp32
 * (values rounded to fp32 inside the fp64 buffers): x0 (also a given one) is
 * rounded to fp32, r is rounded after its computation in u_r, d is rounded and
 * x = fl32(x + d); u_stop defaults to 2^-24 instead of 2^-53.  A: caller CSR
 * (device); b: device fp64; x: device fp64, in/out; M: the unbucketed M for x0
 * (may be NULL when x0_given).  Stopping: nbe <= u_stop, ||d||_inf <= u_stop
 * ||x||_inf, or stagnation.  Returns BSPAI_OK on one of those, else
 * BSPAI_NOT_CONVERGED / BSPAI_NONFINITE / BSPAI_TIMEOUT. */
int gmres_ir_solve(const bspai_csr_t* A, const double* b, bspai_BM_h M_bucketed, bspai_M_h M,
                   bspai_prec_t u, bspai_prec_t u_r, bspai_prec_t u_g, bspai_prec_t u_p,
                   double tol, const bspai_opts_t* opts, double* x, bspai_stream_t s,
                   bspai_solve_info_t* info);

/* ------------------------------------------------------------------ adjoint */
/* Operators for the adjoint system A^T lambda = g (a differentiation
 * extension; Alg 3.1 applied to A^T with the transposed bucketed M as left
 * preconditioner).  Each returns a new library-owned handle:
 *   bspai_matrix_transpose: A^T with the same fp64 / fp32 values (SELL-32);
 *   bspai_M_transpose:      M^T in u_f (for x0 = M^T g);
 *   bspai_bucket_transpose: M^T keeping every entry's bucket and stored value
 *     (fp16 bucket scales unchanged; an e4m3 bucket's per-column scales of M
 *     become per-row scales of M^T), so M^T v is the exact transpose of the
 *     operator bspai_apply uses.  bspai_bucket_export is not available on it.
 * Solve with gmres_ir_solve_h(At, g, BMt, Mt, ...). */
int bspai_matrix_transpose(bspai_A_h A, bspai_stream_t s, bspai_A_h* At);
int bspai_M_transpose(bspai_M_h M, bspai_stream_t s, bspai_M_h* Mt);
int bspai_bucket_transpose(bspai_BM_h BM, bspai_stream_t s, bspai_BM_h* BMt);

/* Gradient of a loss L(x) with respect to the nonzeros of A, where A x_r = b_r
 * for nrhs right-hand sides and lambda_r = A^-T dL/dx_r: dA[p] = sum over r of
 * -lambda_r[i] x_r[j] for the p-th nonzero (i, j) of A's CSR (fp64; r
 * ascending from 0, each product and each sum rounded once).  A: caller CSR
 * (values unused); lambda, x: device fp64, nrhs rows of length n (row r at
 * offset r n); dA: device fp64 length nnz(A), overwritten.  nrhs < 1:
 * BSPAI_ERR_INVALID.  (dL/db_r = lambda_r.) */
int bspai_adjoint_grad_A(const bspai_csr_t* A, int32_t nrhs, const double* lambda, const double* x, double* dA,
                         bspai_stream_t s);

/* ------------------------------------------------------------------ batches */
typedef struct {
    int32_t pairs;          /* nsys * nrhs (system, right-hand side) solves */
    int32_t converged;      /* pairs that met a stopping test */
    int32_t nonfinite;      /* pairs that hit NaN / Inf */
    int32_t ir_launches;    /* refinement steps launched for the batch */
    int32_t max_ir_steps;   /* most GMRES runs of any pair */
    int32_t max_iters;      /* most GMRES steps of any pair, summed over its refinement steps */
    int64_t total_iters;    /* GMRES steps over all pairs */
    int32_t block_threads;  /* CTA size of the schedule used */
    int32_t grid;           /* CTAs of the persistent GMRES launch */
    int32_t kmax;           /* GMRES steps allowed per refinement step */
    int32_t mgs_rows;       /* the schedule's MGS load tile (bspai_batch_schedule_t) */
    int32_t z_shared_rows;  /* the schedule's z-in-shared-memory limit */
    int32_t m_schedule;     /* the schedule's bucket order */
    int32_t team_rows;      /* the schedule's team mode (0: one CTA per pair) */
    int32_t tuned_candidates; /* schedules timed by this call (0: cached or forced) */
    float tune_ms;          /* their summed GPU time */
    int64_t gmres_bytes;    /* algorithmic bytes of the refinement steps' GMRES launches: per
                               Arnoldi step of a pair j + 2 of its vectors (the MGS reads and
                               the new vector), and its two products at the batch's average
                               bytes per row (A in u_p, bucketed M, int32 columns) plus four
                               vectors */
} bspai_batch_info_t;

/* A schedule of the batched GMRES launch.  For a given block_threads every
 * schedule computes the same bits (the dot products of MGS are summed per
 * thread over rows t, t + block_threads, ... and then over the CTA in a fixed
 * tree); the other three fields move loads and storage only.
 *   block_threads  CTA size: 128, 256 or 512 (one CTA per (system, RHS) pair).
 *   mgs_rows       the MGS load tile: rows per thread whose loads one pass
 *                  issues before any arithmetic (u_g fp32: 8 or 16; fp64: 4 or
 *                  8; 0 = the smaller).
 *   z_shared_rows  pairs of at most this many rows keep z, the vector being
 *                  orthogonalised, in shared memory for the whole Arnoldi step
 *                  (0 = never; -1 = as many rows as fit); limited by the
 *                  shared memory left at the CTAs per SM that the registers
 *                  allow.
 *   m_schedule     the bucket schedule of the M products: 0 row-fused (each
 *                  thread takes two rows at a time through every bucket), 1
 *                  bucket-major (one sweep over the pair's rows per bucket,
 *                  the partial sums carried in fp64 between sweeps).
 *   team_rows      0: one CTA per pair (the four fields above).  Otherwise
 *                  (u_g = FP32 only; a multiple of 1024, at most 8192) team
 *                  mode: a pair of n_s rows runs on a team of
 *                  ceil(n_s / team_rows) 512-thread CTAs (at most 32) of one
 *                  cooperative launch in which every team size has a group of
 *                  CTAs in proportion to the sum of n_s^2 of its pairs (a team
 *                  whose group has no pair left takes pairs of the groups of
 *                  smaller pairs), each CTA holding its rows of z and of the
 *                  basis vectors of the current MGS pass in registers; the dot products sum a
 *                  thread's rows, the CTA's threads, then the team's CTAs in
 *                  rank order (other bits than the one-CTA schedules, the same
 *                  in every run).  The other fields are then ignored. */
typedef struct {
    int32_t block_threads;
    int32_t mgs_rows;
    int32_t z_shared_rows;
    int32_t m_schedule;
    int32_t team_rows;
} bspai_batch_schedule_t;

/* Fixes the schedule of later gmres_ir_solve_batched calls made by the calling
 * host thread (NULL: back to the autotuner).  Checked when the solve runs: a
 * field outside its candidates, or z_shared_rows above what fits, gives
 * BSPAI_ERR_INVALID there.  Here only block_threads and m_schedule are checked. */
int bspai_batch_schedule_force(const bspai_batch_schedule_t* sched);

/* The candidates the most recent autotuning (any thread) timed, in the order
 * timed, and the GPU milliseconds of each one's sample run (the largest pairs,
 * four per SM, 32 Arnoldi steps each): up to cap entries
 * into sched / ms (host arrays); *count = the number the tuning timed. */
int bspai_batch_tune_table(bspai_batch_schedule_t* sched, float* ms, int32_t cap, int32_t* count);

/* BSPAI-GMRES-IR (Alg 3.1) for nsys independent systems with nrhs right-hand
 * sides each.  A, the pattern and M hold the systems block-diagonally: system s
 * owns rows row_off[s] .. row_off[s+1]-1 (device int32, nsys + 1 entries,
 * multiples of 32; rows that pad a system have no entries), so one bspai_build
 * and one bspai_bucket_batched call serve the whole batch.  B and X (device
 * fp64) hold nrhs vectors of length n one after another; X is in/out.  Every
 * (system, right-hand side) pair runs its own refinement: per pair x0 = M b
 * (u_f), residuals with u_r ~ u^2 (Dot2), nbe / ||d|| / stagnation tests as in
 * gmres_ir_solve, and its own left-preconditioned MGS-GMRES (vectors in u_g,
 * A v in u_p, bucketed M v, Givens in fp64).  Each refinement step of the
 * batch is one persistent launch in which a CTA takes pairs, largest systems
 * first, and runs each GMRES with CTA barriers only -- or, in team mode, one
 * cooperative launch in which teams of CTAs take pairs.  The schedule (bspai_batch_schedule_t) is chosen by timing
 * candidates on a sample run (the largest pairs, four per SM, 32 Arnoldi
 * steps) in a staged search -- CTA size, then the MGS tile, then z in shared
 * memory, then the bucket schedule, then team mode at 8192 and 4096 rows per
 * CTA (u_g = FP32; tried only when every pair takes the same team size) -- and
 * cached per shape.  The operations of one refinement
 * step (residuals, tests, the GMRES launches, tests) are captured once into a
 * CUDA graph and replayed for every step (launched directly while
 * kernel-class profiling is on, or if the capture fails).  A team exchange
 * that waits longer than opts.barrier_timeout_s gives BSPAI_TIMEOUT.  kmax
 * defaults to
 * min(largest system, 300).  pair_status (0 not converged, 1 nbe, 2 dx,
 * 3 stagnation, -1 non-finite) and pair_iters (device int32, nsys * nrhs,
 * pair p = rhs * nsys + system) may be NULL.  BM must come from
 * bspai_bucket_batched (a bspai_bucket handle, whose buckets use another slot
 * arrangement: BSPAI_ERR_INVALID).  Returns BSPAI_OK when every pair met a
 * stopping test, else BSPAI_NOT_CONVERGED / BSPAI_NONFINITE. */
int gmres_ir_solve_batched(bspai_A_h A, const int32_t* row_off, int32_t nsys, int32_t nrhs, const double* B,
                           bspai_BM_h BM, bspai_M_h M, bspai_prec_t u_g, bspai_prec_t u_p, double tol,
                           const bspai_opts_t* opts, double* X, bspai_stream_t s, bspai_batch_info_t* info,
                           int32_t* pair_status, int32_t* pair_iters);

/* Same as gmres_ir_solve with A already prepared by bspai_matrix_create. */
int gmres_ir_solve_h(bspai_A_h A, const double* b, bspai_BM_h M_bucketed, bspai_M_h M,
                     bspai_prec_t u, bspai_prec_t u_r, bspai_prec_t u_g, bspai_prec_t u_p,
                     double tol, const bspai_opts_t* opts, double* x, bspai_stream_t s,
                     bspai_solve_info_t* info);

/* gmres_ir_solve_h with A v inside GMRES by the adaptive-precision SpMV on A's
 * buckets (bspai_bucket_A; Section 3, eq. nbe2 and fe2).  The residual still
 * uses A's fp64 values in u_r; x0 = M b in u_f; u_p is replaced by the buckets
 * (u_g is used for both).  A_bucketed must hold A's n rows (else
 * BSPAI_ERR_INVALID); precisions, vectors and returns as gmres_ir_solve. */
int gmres_ir_solve_hb(bspai_A_h A, bspai_BM_h A_bucketed, const double* b, bspai_BM_h M_bucketed, bspai_M_h M,
                      bspai_prec_t u, bspai_prec_t u_r, bspai_prec_t u_g, double tol, const bspai_opts_t* opts,
                      double* x, bspai_stream_t s, bspai_solve_info_t* info);

#ifdef __cplusplus
}
#endif
#endif /* BSPAI_H */
