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

namespace bspai {

template <typename XT>
__device__ __forceinline__ float to_f32(XT v);
template <>
__device__ __forceinline__ float to_f32<double>(double v) { return __double2float_rn(v); }
template <>
__device__ __forceinline__ float to_f32<float>(float v) { return v; }

template <typename YT>
__device__ __forceinline__ YT from_f64(double v);
template <>
__device__ __forceinline__ double from_f64<double>(double v) { return v; }
template <>
__device__ __forceinline__ float from_f64<float>(double v) { return __double2float_rn(v); }

// Decode one stored value of a narrow bucket to fp32 (exact: the scales are
// powers of two and the narrow formats embed in fp32).
template <int PREC>
__device__ __forceinline__ float decode(const void* val, int64_t p, float scale, const float* colscale, int c);
template <>
__device__ __forceinline__ float decode<BSPAI_FP32>(const void* val, int64_t p, float, const float*, int) {
    return __ldg(reinterpret_cast<const float*>(val) + p);
}
template <>
__device__ __forceinline__ float decode<BSPAI_FP16>(const void* val, int64_t p, float scale, const float*, int) {
    return __fmul_rn(__half2float(reinterpret_cast<const __half*>(val)[p]), scale);
}
template <>
__device__ __forceinline__ float decode<BSPAI_BF16>(const void* val, int64_t p, float, const float*, int) {
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(val)[p]);
}
template <>
__device__ __forceinline__ float decode<BSPAI_E4M3>(const void* val, int64_t p, float, const float* colscale, int c) {
    __nv_fp8_e4m3 e;
    e.__x = reinterpret_cast<const __nv_fp8_storage_t*>(val)[p];
    return __fmul_rn(float(e), __ldg(colscale + c));
}

// fp32 partial sum of one row over one narrow bucket.  Loads are issued four
// slots ahead of the (strictly sequential) accumulation.
template <int PREC, typename XT>
__device__ __forceinline__ float row_partial_f32(const BucketDev& B, int64_t p, int64_t end,
                                                 const XT* __restrict__ x) {
    float acc = 0.0f;
    for (; p + 96 < end; p += 128) {
        int c[4];
        float v[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) c[u] = __ldg(B.col + p + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (c[u] >= 0) {
                v[u] = decode<PREC>(B.val, p + 32 * u, B.scale, B.colscale, c[u]);
                xv[u] = to_f32<XT>(__ldg(x + c[u]));
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (c[u] >= 0) acc = __fadd_rn(acc, __fmul_rn(v[u], xv[u]));
    }
    for (; p < end; p += 32) {
        int c = __ldg(B.col + p);
        if (c >= 0) {
            float v = decode<PREC>(B.val, p, B.scale, B.colscale, c);
            acc = __fadd_rn(acc, __fmul_rn(v, to_f32<XT>(__ldg(x + c))));
        }
    }
    return acc;
}

template <typename XT>
__device__ __forceinline__ double row_partial_f64(const BucketDev& B, int64_t p, int64_t end,
                                                  const XT* __restrict__ x) {
    const double* val = reinterpret_cast<const double*>(B.val);
    double acc = 0.0;
    for (; p + 96 < end; p += 128) {
        int c[4];
        double v[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) c[u] = __ldg(B.col + p + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (c[u] >= 0) {
                v[u] = __ldg(val + p + 32 * u);
                xv[u] = (double)__ldg(x + c[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (c[u] >= 0) acc = __dadd_rn(acc, __dmul_rn(v[u], xv[u]));
    }
    for (; p < end; p += 32) {
        int c = __ldg(B.col + p);
        if (c >= 0) acc = __dadd_rn(acc, __dmul_rn(__ldg(val + p), (double)__ldg(x + c)));
    }
    return acc;
}

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
    double yi = 0.0;
    for (int k = 0; k < M.q; ++k) {
        const BucketDev& B = M.b[k];
        const int64_t p0 = B.sptr[s] + lane;
        const int64_t end = B.sptr[s + 1];
        switch (B.prec) {
        case BSPAI_FP64: yi = __dadd_rn(yi, row_partial_f64<XT>(B, p0, end, x)); break;
        case BSPAI_FP32: yi = __dadd_rn(yi, (double)row_partial_f32<BSPAI_FP32, XT>(B, p0, end, x)); break;
        case BSPAI_FP16: yi = __dadd_rn(yi, (double)row_partial_f32<BSPAI_FP16, XT>(B, p0, end, x)); break;
        case BSPAI_BF16: yi = __dadd_rn(yi, (double)row_partial_f32<BSPAI_BF16, XT>(B, p0, end, x)); break;
        case BSPAI_E4M3: yi = __dadd_rn(yi, (double)row_partial_f32<BSPAI_E4M3, XT>(B, p0, end, x)); break;
        default: break;  // dropped entries are not stored
        }
    }
    if (r < M.n) y[r] = from_f64<YT>(yi);
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
    return d;
}

int launch_bspmv_idx(const BMDev& M, const void* x, int x_prec, void* y, int y_prec, const int* jd,
                     int64_t ldx, int64_t ldy, int yoff, cudaStream_t s) {
    if (M.n == 0) return BSPAI_OK;
    const int64_t rows = ceil_div(M.n, kSlice) * kSlice;
    const unsigned grid = (unsigned)ceil_div(rows, 256);
    if (x_prec == BSPAI_FP64 && y_prec == BSPAI_FP64)
        k_bspmv<double, double><<<grid, 256, 0, s>>>(M, (const double*)x, (double*)y, jd, ldx, ldy, yoff);
    else if (x_prec == BSPAI_FP64 && y_prec == BSPAI_FP32)
        k_bspmv<double, float><<<grid, 256, 0, s>>>(M, (const double*)x, (float*)y, jd, ldx, ldy, yoff);
    else if (x_prec == BSPAI_FP32 && y_prec == BSPAI_FP64)
        k_bspmv<float, double><<<grid, 256, 0, s>>>(M, (const float*)x, (double*)y, jd, ldx, ldy, yoff);
    else if (x_prec == BSPAI_FP32 && y_prec == BSPAI_FP32)
        k_bspmv<float, float><<<grid, 256, 0, s>>>(M, (const float*)x, (float*)y, jd, ldx, ldy, yoff);
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
