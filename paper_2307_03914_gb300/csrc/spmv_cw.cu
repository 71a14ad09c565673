// spmv_cw.cu -- the componentwise, x-dependent bucketed product: the strategy
// of Graillat et al. that Section 2.3 of the paper mentions and sets aside,
// because its buckets depend on the vector x and must be formed again for
// every product.  Built here as a study of that cost.
//
// Reading of the rule (the paper does not print it): for row i,
// s_i = (|M||x|)_i, and entry (i, j) goes to bucket k by the intervals of
// eq. (nint) with |m_ij| |x_j| in place of |m_ij| and s_i in place of ||M||:
//   bucket 0      if |m x| > t_1,
//   bucket q-1    if |m x| <= t_{q-1},
//   bucket k      if t_{k+1} < |m x| <= t_k,      t_k = eps s_i / u_k.
// The product itself is Alg 2.3 on those buckets, in the decoupled form of
// the normwise path (fp64 bucket in fp64, narrow buckets stored in their
// format and accumulated in fp32 with x rounded to fp32, partial sums added
// in fp64 in bucket order).
//
// One thread per row of M's own sliced-ELL structure (its u_f values):
// pass 1 forms s_i (fp64, ascending columns) and the thresholds, pass 2 (the
// row again, from L1) classifies every product and adds it to its bucket's
// partial sum.  There is no stored bucketed matrix: every product reads M in
// u_f, which is the storage the normwise buckets save.  Formats whose range
// needs a scale fitted to the bucket's contents (fp16, e4m3) would need one
// more pass per product and are not offered.
#include "common.cuh"
#include "spmv_row.cuh"

namespace bspai {

struct CwParams {
    int32_t q;
    int32_t precs[4];
    double eps;
    double uk_inv[4];  // 1 / u_k: a power of two, so eps s / u_k = (eps s) (1 / u_k) exactly
};

// a > b for non-negative doubles, by their bit patterns (the integer pipe)
__device__ __forceinline__ bool gt_nonneg(double a, double b) {
    return __double_as_longlong(a) > __double_as_longlong(b);
}

constexpr int kCwCache = 8;  // products |m x| of a row's first slots kept in registers between the passes

template <typename XT, typename YT>
__global__ void __launch_bounds__(256) k_bspmv_cw(int n, const int64_t* __restrict__ sptr,
                                                  const int32_t* __restrict__ col, const float* __restrict__ val,
                                                  const int32_t* __restrict__ rowlen,
                                                  const int32_t* __restrict__ csr_row_ptr,
                                                  const __grid_constant__ CwParams P, const XT* __restrict__ x,
                                                  YT* __restrict__ y, int8_t* __restrict__ ids,
                                                  unsigned long long* __restrict__ nnzk) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int cnt[4] = {0, 0, 0, 0};
    if (r < n) {
        const int64_t b = sptr[r >> 5] + (r & 31);
        const int len = rowlen[r];
        // pass 1: s_i = (|M||x|)_i in fp64, ascending columns
        double si = 0.0;
        double am[kCwCache];
#pragma unroll
        for (int l = 0; l < kCwCache; ++l) {
            am[l] = 0.0;
            if (l < len) {
                const int64_t p = b + ((int64_t)l << 5);
                am[l] = __dmul_rn(fabs((double)__ldg(val + p)), fabs((double)__ldg(x + __ldg(col + p))));
                si = __dadd_rn(si, am[l]);
            }
        }
        for (int l = kCwCache; l < len; ++l) {
            const int64_t p = b + ((int64_t)l << 5);
            si = __dadd_rn(si, __dmul_rn(fabs((double)__ldg(val + p)), fabs((double)__ldg(x + __ldg(col + p)))));
        }
        double thr[4];
        thr[0] = __longlong_as_double(0x7ff0000000000000LL);
        const double es = __dmul_rn(P.eps, si);
#pragma unroll
        for (int k = 1; k < 4; ++k) thr[k] = k < P.q ? __dmul_rn(es, P.uk_inv[k]) : 0.0;
        // pass 2: the bucket of every product, and the bucket partial sums
        double acc64 = 0.0;
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        const int o = csr_row_ptr ? csr_row_ptr[r] : 0;
        for (int l = 0; l < len; ++l) {
            const int64_t p = b + ((int64_t)l << 5);
            const float m = __ldg(val + p);
            const XT xv = __ldg(x + __ldg(col + p));
            double a = 0.0;
#pragma unroll
            for (int c = 0; c < kCwCache; ++c)
                if (c == l) a = am[c];
            if (l >= kCwCache) a = __dmul_rn(fabs((double)m), fabs((double)xv));
            int k = 0;
            if (P.q == 1 || gt_nonneg(a, thr[1])) {
                k = 0;
            } else if (!gt_nonneg(a, thr[P.q - 1])) {
                k = P.q - 1;
            } else {
                for (int bb = 1; bb <= P.q - 2; ++bb)
                    if (gt_nonneg(a, thr[bb + 1]) && !gt_nonneg(a, thr[bb])) k = bb;
            }
            if (ids) ids[o + l] = (int8_t)k;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                if (kk != k) continue;
                cnt[kk] += 1;
                switch (P.precs[kk]) {
                case BSPAI_FP64: acc64 = __dadd_rn(acc64, __dmul_rn((double)m, (double)xv)); break;
                case BSPAI_FP32: acc[kk] = __fadd_rn(acc[kk], __fmul_rn(m, to_f32<XT>(xv))); break;
                case BSPAI_BF16:
                    acc[kk] = __fadd_rn(acc[kk], __fmul_rn(__bfloat162float(__float2bfloat16_rn(m)), to_f32<XT>(xv)));
                    break;
                default: break;  // dropped
                }
            }
        }
        double yi = 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (k >= P.q) break;
            if (P.precs[k] == BSPAI_FP64) yi = __dadd_rn(yi, acc64);
            else if (P.precs[k] != BSPAI_DROP) yi = __dadd_rn(yi, (double)acc[k]);
        }
        y[r] = from_f64<YT>(yi);
    }
    if (nnzk) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int c = cnt[k];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
            if ((threadIdx.x & 31) == 0 && c) atomicAdd(nnzk + k, (unsigned long long)c);
        }
    }
}

}  // namespace bspai

using namespace bspai;

extern "C" {

int bspai_apply_cw(bspai_M_h M, double bucket_eps, const int32_t* precs, int32_t q, const void* x,
                   bspai_prec_t x_prec, void* y, bspai_prec_t y_prec, int8_t* ids, int64_t* nnz_k,
                   bspai_stream_t st) {
    cudaStream_t s = (cudaStream_t)st;
    if (!M || M->magic != kMagicM) return set_error(BSPAI_ERR_INVALID, "bspai_apply_cw: bad handle");
    if (!precs || q < 1 || q > 4) return set_error(BSPAI_ERR_INVALID, "bspai_apply_cw: need 1 <= q <= 4 precisions");
    if (!(bucket_eps > 0.0)) return set_error(BSPAI_ERR_INVALID, "bspai_apply_cw: bucket_eps must be > 0");
    if (M->n > 0 && (!x || !y)) return set_error(BSPAI_ERR_INVALID, "bspai_apply_cw: null vector");
    if (ids && !M->csr_row_ptr)
        return set_error(BSPAI_ERR_INVALID, "bspai_apply_cw: this handle keeps no CSR row pointers for ids");
    CwParams P{};
    P.q = q;
    P.eps = bucket_eps;
    for (int k = 0; k < q; ++k) {
        const int f = precs[k];
        if (f != BSPAI_FP64 && f != BSPAI_FP32 && f != BSPAI_BF16 && f != BSPAI_DROP)
            return set_error(BSPAI_ERR_UNSUPPORTED,
                             "bspai_apply_cw: buckets in fp64, fp32, bf16 or drop only (fp16 and e4m3 need a scale "
                             "fitted to each bucket's contents, one more pass per product)");
        P.precs[k] = f;
        P.uk_inv[k] = 1.0 / unit_roundoff(f);
        if (k > 0 && !(unit_roundoff(f) > unit_roundoff(P.precs[k - 1])))
            return set_error(BSPAI_ERR_INVALID, "bspai_apply_cw: precisions must have increasing unit roundoff");
    }
    if ((x_prec != BSPAI_FP64 && x_prec != BSPAI_FP32) || (y_prec != BSPAI_FP64 && y_prec != BSPAI_FP32))
        return set_error(BSPAI_ERR_UNSUPPORTED, "bspai_apply_cw: x and y must be FP64 or FP32");
    if (M->n == 0) return BSPAI_OK;
    unsigned long long* d_cnt = nullptr;
    if (nnz_k) {
        BSPAI_TRY(dalloc_t(&d_cnt, 4, s));
        CUDA_TRY(cudaMemsetAsync(d_cnt, 0, 4 * sizeof(unsigned long long), s));
    }
    ProfScope ps(BSPAI_K_BSPMV, s);
    const unsigned grid = (unsigned)ceil_div(M->n, 256);
    const Sell& S = M->sell;
    if (x_prec == BSPAI_FP64 && y_prec == BSPAI_FP64)
        k_bspmv_cw<double, double><<<grid, 256, 0, s>>>(M->n, S.sptr, S.col, M->val, M->rowlen, M->csr_row_ptr, P,
                                                        (const double*)x, (double*)y, ids, d_cnt);
    else if (x_prec == BSPAI_FP64)
        k_bspmv_cw<double, float><<<grid, 256, 0, s>>>(M->n, S.sptr, S.col, M->val, M->rowlen, M->csr_row_ptr, P,
                                                       (const double*)x, (float*)y, ids, d_cnt);
    else if (y_prec == BSPAI_FP64)
        k_bspmv_cw<float, double><<<grid, 256, 0, s>>>(M->n, S.sptr, S.col, M->val, M->rowlen, M->csr_row_ptr, P,
                                                       (const float*)x, (double*)y, ids, d_cnt);
    else
        k_bspmv_cw<float, float><<<grid, 256, 0, s>>>(M->n, S.sptr, S.col, M->val, M->rowlen, M->csr_row_ptr, P,
                                                      (const float*)x, (float*)y, ids, d_cnt);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        dfree(d_cnt, s);
        return cuda_error(e, "k_bspmv_cw", __FILE__, __LINE__);
    }
    if (nnz_k) {
        unsigned long long h[4] = {0, 0, 0, 0};
        e = cudaMemcpyAsync(h, d_cnt, sizeof h, cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        dfree(d_cnt, s);
        if (e) return cuda_error(e, "bspai_apply_cw counts", __FILE__, __LINE__);
        for (int k = 0; k < q; ++k) nnz_k[k] = (int64_t)h[k];
    }
    return BSPAI_OK;
}

}  // extern "C"
