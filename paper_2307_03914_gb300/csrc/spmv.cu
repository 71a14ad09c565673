// spmv.cu -- the adaptive-precision SpMV (Alg 2.3) on SELL-32 buckets, and its
// single-bucket uses: x0 = M b in u_f (Alg 3.1) and A v in u_p.
//
// One thread per row, one warp per 32-row slice.  For each bucket k the row's
// partial sum y_i^(k) is accumulated sequentially in ascending column order:
// in fp64 for an fp64 bucket, in fp32 for fp32/fp16/bf16/e4m3 buckets (storage
// precision u_k, compute precision fp32: the decoupled form the paper names as
// future work in Section 5).  The partial sums are added in fp64 in bucket
// order.  Products and sums use explicit round-to-nearest intrinsics so that
// no fused multiply-add changes the rounding of the textbook model.
#include "common.cuh"
#include "spmv_row.cuh"

namespace bspai {

// `jd` (optional) points at a device pair {j, done} of a running GMRES: the
// kernel does nothing once done is set, and otherwise reads x from column j
// and writes y to column j + yoff of column-major bases (leading dims ldx, ldy).
template <typename XT, typename YT>
__global__ void __launch_bounds__(256) k_bspmv(const __grid_constant__ BMDev M, const XT* __restrict__ x,
                                               YT* __restrict__ y, const int* __restrict__ jd, int64_t ldx,
                                               int64_t ldy, int yoff) {
    if (jd) {
        if (jd[1]) return;
        const int64_t j = jd[0];
        x += j * ldx;
        y += (j + yoff) * ldy;
    }
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s = r >> 5;
    const int lane = (int)(r & 31);
    if (r >= (int64_t)ceil_div(M.n, kSlice) * kSlice) return;
    const double yi = bucketed_row<XT>(M, r, x);
    if (r < M.n) y[r] = from_f64<YT>(yi);
}

// The same product as k_bspmv for Q non-empty buckets, organised for memory-
// level parallelism: the slice bounds of all buckets, then the first W column
// indices of every bucket, then all their values and x entries are loaded
// before any arithmetic, and only then is each bucket's partial sum formed in
// ascending column order (slots beyond W follow in a plain loop) and the
// partial sums added in bucket order.  Identical operations in identical order,
// hence identical bits.  F64: bucket 0 is the fp64 bucket.
template <typename XT, typename YT, int Q, int W, bool F64>
__global__ void __launch_bounds__(256) k_bspmv_q(const __grid_constant__ BMDev M, const XT* __restrict__ x,
                                                 YT* __restrict__ y, const int* __restrict__ jd, int64_t ldx,
                                                 int64_t ldy, int yoff) {
    if (jd) {
        if (jd[1]) return;
        const int64_t j = jd[0];
        x += j * ldx;
        y += (j + yoff) * ldy;
    }
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s = r >> 5;
    const int lane = (int)(r & 31);
    if (r >= (int64_t)ceil_div(M.n, kSlice) * kSlice) return;
    int64_t base[Q];
    int w[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        base[k] = __ldg(M.b[k].sptr + s) + lane;
        w[k] = (int)((__ldg(M.b[k].sptr + s + 1) - (base[k] - lane)) >> 5);
    }
    int c[Q][W];
#pragma unroll
    for (int k = 0; k < Q; ++k)
#pragma unroll
        for (int l = 0; l < W; ++l) c[k][l] = l < w[k] ? __ldg(M.b[k].col + base[k] + 32 * l) : -1;
    float v[Q][W], xf[Q][W];
    double vd[W], xd[W];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
#pragma unroll
        for (int l = 0; l < W; ++l) {
            const int cc = c[k][l];
            if (cc >= 0) {
                if (F64 && k == 0) {
                    vd[l] = __ldg(reinterpret_cast<const double*>(M.b[0].val) + base[0] + 32 * l);
                    xd[l] = (double)__ldg(x + cc);
                } else {
                    v[k][l] = decode_rt(M.b[k], base[k] + 32 * l, cc, r);
                    xf[k][l] = to_f32<XT>(__ldg(x + cc));
                }
            }
        }
    }
    double yi = 0.0;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const BucketDev& B = M.b[k];
        if (F64 && k == 0) {
            double acc = 0.0;
#pragma unroll
            for (int l = 0; l < W; ++l)
                if (c[k][l] >= 0) acc = __dadd_rn(acc, __dmul_rn(vd[l], xd[l]));
            for (int l = W; l < w[k]; ++l) {
                const int cc = __ldg(B.col + base[k] + 32 * l);
                if (cc >= 0)
                    acc = __dadd_rn(acc, __dmul_rn(__ldg(reinterpret_cast<const double*>(B.val) + base[k] + 32 * l),
                                                   (double)__ldg(x + cc)));
            }
            yi = __dadd_rn(yi, acc);
        } else {
            float acc = 0.0f;
#pragma unroll
            for (int l = 0; l < W; ++l)
                if (c[k][l] >= 0) acc = __fadd_rn(acc, __fmul_rn(v[k][l], xf[k][l]));
            for (int l = W; l < w[k]; ++l) {
                const int cc = __ldg(B.col + base[k] + 32 * l);
                if (cc >= 0) acc = __fadd_rn(acc, __fmul_rn(decode_rt(B, base[k] + 32 * l, cc, r), to_f32<XT>(__ldg(x + cc))));
            }
            yi = __dadd_rn(yi, (double)acc);
        }
    }
    if (r < M.n) y[r] = from_f64<YT>(yi);
}

template <typename XT, typename YT>
using BspmvFn = void (*)(BMDev, const XT*, YT*, const int*, int64_t, int64_t, int);

// pick the k_bspmv_q instance for (Q, W, F64); null if none fits
template <typename XT, typename YT>
static BspmvFn<XT, YT> pick_q(int Q, int W, bool f64) {
#define BSPAI_PICK(q, w)                                                                  \
    if (Q == q && W == w) return f64 ? (BspmvFn<XT, YT>)k_bspmv_q<XT, YT, q, w, true>      \
                                     : (BspmvFn<XT, YT>)k_bspmv_q<XT, YT, q, w, false>;
    BSPAI_PICK(1, 4) BSPAI_PICK(1, 8) BSPAI_PICK(2, 4) BSPAI_PICK(2, 8) BSPAI_PICK(3, 4) BSPAI_PICK(4, 4)
#undef BSPAI_PICK
    return nullptr;
}

BMDev single_bucket_view(const Sell& S, const void* val, int prec) {
    BMDev d{};
    d.n = S.n;
    d.q = 1;
    d.b[0].prec = prec;
    d.b[0].scale = 1.0f;
    d.b[0].sptr = S.sptr;
    d.b[0].col = S.col;
    d.b[0].val = val;
    d.b[0].colscale = nullptr;
    d.b[0].rowscale = nullptr;
    d.b[0].slicescale = nullptr;
    d.b[0].nnz = -1;
    d.b[0].maxw = -1;
    return d;
}

// Buckets that contribute nothing (dropped, or with no entries) are left out:
// their partial sums are +0 and adding +0 to a sum that is never -0 changes nothing.
static BMDev compact_buckets(const BMDev& M) {
    BMDev c = M;
    c.q = 0;
    for (int k = 0; k < M.q; ++k)
        if (M.b[k].prec != BSPAI_DROP && M.b[k].nnz != 0) c.b[c.q++] = M.b[k];
    return c;
}

template <typename XT, typename YT>
static void launch_typed(const BMDev& M0, const XT* x, YT* y, const int* jd, int64_t ldx, int64_t ldy, int yoff,
                         unsigned grid, cudaStream_t s) {
    const BMDev M = compact_buckets(M0);
    int maxw = 0;
    bool known = true;
    for (int k = 0; k < M.q; ++k) {
        if (M.b[k].maxw < 0) known = false;
        maxw = M.b[k].maxw > maxw ? M.b[k].maxw : maxw;
    }
    const int W = (M.q <= 2 && (!known || maxw > 4)) ? 8 : 4;
    BspmvFn<XT, YT> fn = M.q >= 1 ? pick_q<XT, YT>(M.q, W, M.b[0].prec == BSPAI_FP64) : nullptr;
    if (fn)
        fn<<<grid, 256, 0, s>>>(M, x, y, jd, ldx, ldy, yoff);
    else
        k_bspmv<XT, YT><<<grid, 256, 0, s>>>(M, x, y, jd, ldx, ldy, yoff);
}

int launch_bspmv_idx(const BMDev& M, const void* x, int x_prec, void* y, int y_prec, const int* jd,
                     int64_t ldx, int64_t ldy, int yoff, cudaStream_t s) {
    if (M.n == 0) return BSPAI_OK;
    const int64_t rows = ceil_div(M.n, kSlice) * kSlice;
    const unsigned grid = (unsigned)ceil_div(rows, 256);
    if (x_prec == BSPAI_FP64 && y_prec == BSPAI_FP64)
        launch_typed<double, double>(M, (const double*)x, (double*)y, jd, ldx, ldy, yoff, grid, s);
    else if (x_prec == BSPAI_FP64 && y_prec == BSPAI_FP32)
        launch_typed<double, float>(M, (const double*)x, (float*)y, jd, ldx, ldy, yoff, grid, s);
    else if (x_prec == BSPAI_FP32 && y_prec == BSPAI_FP64)
        launch_typed<float, double>(M, (const float*)x, (double*)y, jd, ldx, ldy, yoff, grid, s);
    else if (x_prec == BSPAI_FP32 && y_prec == BSPAI_FP32)
        launch_typed<float, float>(M, (const float*)x, (float*)y, jd, ldx, ldy, yoff, grid, s);
    else
        return set_error(BSPAI_ERR_UNSUPPORTED, "bspmv: x/y precision must be FP64 or FP32");
    note_launch();
    CUDA_LAUNCH_CHECK();
    return BSPAI_OK;
}

int launch_bspmv(const BMDev& M, const void* x, int x_prec, void* y, int y_prec, cudaStream_t s) {
    return launch_bspmv_idx(M, x, x_prec, y, y_prec, nullptr, 0, 0, 0, s);
}

}  // namespace bspai

using namespace bspai;

BMDev bspai_bucketed::dev() const {
    BMDev d{};
    d.n = n;
    d.q = q;
    for (int k = 0; k < q; ++k) {
        d.b[k].prec = precs[k];
        d.b[k].scale = scale[k];
        d.b[k].sptr = b[k].sptr;
        d.b[k].col = b[k].col;
        d.b[k].val = val[k];
        d.b[k].colscale = precs[k] == BSPAI_E4M3 ? colscale : nullptr;
        d.b[k].rowscale = precs[k] == BSPAI_E4M3 ? rowscale : nullptr;
        d.b[k].slicescale = sscale[k];
        d.b[k].nnz = nnz_k[k];
        d.b[k].maxw = maxw[k];
    }
    return d;
}

extern "C" {

int bspai_apply(bspai_BM_h BM, const void* x, bspai_prec_t x_prec, void* y, bspai_prec_t y_prec,
                bspai_stream_t s) {
    if (!BM || BM->magic != kMagicBM) return set_error(BSPAI_ERR_INVALID, "bspai_apply: bad handle");
    if (!x || !y) return set_error(BSPAI_ERR_INVALID, "bspai_apply: null vector");
    ProfScope ps(BSPAI_K_BSPMV, (cudaStream_t)s);
    return launch_bspmv(BM->dev(), x, x_prec, y, y_prec, (cudaStream_t)s);
}

int bspai_apply_uf(bspai_M_h M, const double* x, double* y, bspai_stream_t s) {
    if (!M || M->magic != kMagicM) return set_error(BSPAI_ERR_INVALID, "bspai_apply_uf: bad handle");
    if (!x || !y) return set_error(BSPAI_ERR_INVALID, "bspai_apply_uf: null vector");
    ProfScope ps(BSPAI_K_OTHER, (cudaStream_t)s);
    return launch_bspmv(single_bucket_view(M->sell, M->val, BSPAI_FP32), x, BSPAI_FP64, y, BSPAI_FP64,
                        (cudaStream_t)s);
}

int bspai_spmv_up(bspai_A_h A, const float* v, float* w, bspai_stream_t s) {
    if (!A || A->magic != kMagicA) return set_error(BSPAI_ERR_INVALID, "bspai_spmv_up: bad handle");
    if (!v || !w) return set_error(BSPAI_ERR_INVALID, "bspai_spmv_up: null vector");
    ProfScope ps(BSPAI_K_SPMV_A, (cudaStream_t)s);
    return launch_bspmv(single_bucket_view(A->sell, A->val32, BSPAI_FP32), v, BSPAI_FP32, w, BSPAI_FP32,
                        (cudaStream_t)s);
}

}  // extern "C"
