// bucket.cu -- precision buckets of M (eq. nint, Alg 2.2) and their storage;
// the same bucketing applied to A (fp64 values) for the bucketed A v.
//
// ||M||_inf is the max over rows of the fp64 sum of |m_ij| taken in ascending
// column order (one thread per row), so it and the thresholds
// t_k = eps ||M||_inf / u_k are bit-for-bit reproducible.  Each entry goes to
//   bucket 0      if |m| > t_1,
//   bucket q-1    if |m| <= t_{q-1},
//   bucket k      if t_{k+1} < |m| <= t_k   (0 < k < q-1),
// boundary values to the lower-precision bucket.  Every bucket gets its own
// SELL-32 structure (entries of a row keep their ascending column order);
// values are stored in the bucket's format: fp16 with one power-of-two scale
// per bucket, e4m3 with a power-of-two fp32 scale per column, so that the
// narrow formats' exponent range does not flush the small entries.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace bspai {

double unit_roundoff(int prec) {
    switch (prec) {
    case BSPAI_FP64: return 0x1p-53;
    case BSPAI_FP32: return 0x1p-24;
    case BSPAI_FP16: return 0x1p-11;
    case BSPAI_BF16: return 0x1p-8;
    case BSPAI_E4M3: return 0x1p-4;
    case BSPAI_DROP: return 1.0;
    default: return -1.0;
    }
}

static int prec_bits(int prec) {
    switch (prec) {
    case BSPAI_FP64: return 64;
    case BSPAI_FP32: return 32;
    case BSPAI_FP16: return 16;
    case BSPAI_BF16: return 16;
    case BSPAI_E4M3: return 8;
    default: return 0;
    }
}

static size_t prec_bytes(int prec) { return (size_t)prec_bits(prec) / 8; }

struct BucketParams {
    int32_t q;
    int32_t precs[8];
    double eps;
    double uk[8];
};

struct PackDst {
    int32_t q;
    int32_t precs[8];
    int64_t* sptr[8];
    int32_t* col[8];     // int32 columns, or null when col16 is used
    int16_t* col16[8];   // 16-bit column differences c - r, or null
    void* val[8];
    float scale[8];
    int32_t packed;      // slot arrangement of every bucket (Sell::packed)
};

// In a batch of independent systems stacked block-diagonally, every 32-row
// slice belongs to one system (slice_seg[s]); each system gets its own
// ||M_s||_inf, thresholds and fp16 scales, exactly as if it were bucketed
// alone.  slice_seg = null means one system.
__device__ __forceinline__ int seg_of(const int32_t* slice_seg, int64_t slice) {
    return slice_seg ? slice_seg[slice] : 0;
}

template <typename VT>
__global__ void k_norm_rows(int n, const int64_t* __restrict__ sptr, const VT* __restrict__ val,
                            const int32_t* __restrict__ rowlen, const int32_t* __restrict__ slice_seg,
                            double* __restrict__ norm) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (r < n) {
        const int64_t b = sptr[r >> 5] + (r & 31);
        const int len = rowlen[r];
        for (int l = 0; l < len; ++l) s = __dadd_rn(s, fabs((double)val[b + (int64_t)l * kSlice]));
    }
    // the warp's rows form one slice (one segment): one atomic per warp
    s = warp_max_bits(s);
    if ((threadIdx.x & 31) == 0 && r < n && s != 0.0) atomic_max_nonneg(norm + seg_of(slice_seg, r >> 5), s);
}

__global__ void k_thresholds(const __grid_constant__ BucketParams P, int nseg, const double* __restrict__ norm,
                             double* __restrict__ thr) {
    const int sg = blockIdx.x * blockDim.x + threadIdx.x;
    if (sg >= nseg) return;
    thr[sg * 8] = __longlong_as_double(0x7ff0000000000000LL);
    for (int k = 1; k < P.q; ++k) thr[sg * 8 + k] = __ddiv_rn(__dmul_rn(P.eps, norm[sg]), P.uk[k]);
}

__device__ __forceinline__ int classify(double a, const double* thr, int q) {
    if (q == 1 || a > thr[1]) return 0;
    if (a <= thr[q - 1]) return q - 1;
    int k = 0;
    for (int b = 1; b <= q - 2; ++b)
        if (a > thr[b + 1] && a <= thr[b]) k = b;
    return k;
}

// one row of k_classify (a live warp's rows): ids, per-slice widths, and the
// warp's contributions to the block's counts and maxima
template <typename VT>
__device__ __forceinline__ void classify_rows(int64_t r, int n, int nslices, const int64_t* __restrict__ sptr,
                                              const int32_t* __restrict__ col, const VT* __restrict__ val,
                                              const int32_t* __restrict__ rowlen, const BucketParams& P,
                                              const double* __restrict__ thr_g, int8_t* __restrict__ id,
                                              int64_t* __restrict__ widths, VT* __restrict__ colmax,
                                              const int32_t* __restrict__ slice_seg, int packed,
                                              VT* __restrict__ bmax, bool one_seg, unsigned long long* s_cnt,
                                              int* s_wmax, int* s_wmin, VT* s_bmax, unsigned* s_dmax) {
    unsigned dm = 0;  // max |c - r| of the row
    const int sg = seg_of(slice_seg, r >> 5);
    double thr[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) thr[k] = k < P.q ? thr_g[sg * 8 + k] : 0.0;
    int cnt[8];
    VT mx[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        cnt[k] = 0;
        mx[k] = VT(0);
    }
    if (r < n) {
        const int64_t b = sptr[r >> 5] + (r & 31);
        const int len = rowlen[r];
        for (int l = 0; l < len; ++l) {
            const int64_t slot = b + (int64_t)l * kSlice;
            const VT m = val[slot];
            const VT am = fabs(m);
            const int k = classify((double)am, thr, P.q);
            id[slot] = (int8_t)k;
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                if (kk == k) {
                    cnt[kk] += 1;
                    mx[kk] = fmax(mx[kk], am);
                }
            }
            if (P.precs[k] == BSPAI_E4M3) atomic_max_nonneg(colmax + col[slot], am);
            const int64_t d = (int64_t)col[slot] - r;
            const unsigned ad = (unsigned)(d < 0 ? (d < -0x7fffffff ? 0x7fffffff : -d) : (d > 0x7fffffff ? 0x7fffffff : d));
            dm = ad > dm ? ad : dm;
        }
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned t = __shfl_xor_sync(0xffffffffu, dm, o);
        dm = t > dm ? t : dm;
    }
    if (lane == 0 && dm) atomicMax(s_dmax, dm);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (k >= P.q) break;
        int w = cnt[k], c = cnt[k];
        VT m = mx[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            w = max(w, __shfl_xor_sync(0xffffffffu, w, o));
            c += __shfl_xor_sync(0xffffffffu, c, o);
            m = fmax(m, (VT)__shfl_xor_sync(0xffffffffu, m, o));
        }
        if (packed) w = (w + 3) & ~3;  // groups of four slots per row
        if (lane == 0) {
            widths[(int64_t)k * (nslices + 1) + (r >> 5)] = (int64_t)w * kSlice;
            if (c) atomicAdd(s_cnt + k, (unsigned long long)c);
            if (m > VT(0)) atomic_max_nonneg(one_seg ? s_bmax + k : bmax + sg * 8 + k, m);
            if (w) atomicMax(s_wmax + k, w);
            atomicMin(s_wmin + k, w);
        }
    }
}


// bucket id of every entry; per-slice widths of every bucket; per-bucket
// counts and max |m|; per-column max |m| of the e4m3 bucket
template <typename VT>
__global__ void __launch_bounds__(256) k_classify(int n, int nslices, const int64_t* __restrict__ sptr,
                                                  const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                  const int32_t* __restrict__ rowlen,
                                                  const __grid_constant__ BucketParams P,
                                                  const double* __restrict__ thr_g, int8_t* __restrict__ id,
                                                  int64_t* __restrict__ widths, unsigned long long* __restrict__ nnzk,
                                                  VT* __restrict__ bmax, VT* __restrict__ colmax,
                                                  int* __restrict__ wmax, const int32_t* __restrict__ slice_seg,
                                                  int packed, unsigned* __restrict__ dmax, int* __restrict__ wmin) {
    // the warps' counts, widths and maxima meet in shared memory first: one
    // global atomic per block and quantity instead of one per warp (max, min and
    // integer sums: the totals do not depend on the order)
    __shared__ unsigned long long s_cnt[8];
    __shared__ int s_wmax[8], s_wmin[8];
    __shared__ __align__(8) unsigned s_bmax[8 * (sizeof(VT) / 4)];
    __shared__ unsigned s_dmax;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t rows = (int64_t)nslices * kSlice;
    const bool live = r < rows;  // whole warps (rows is a multiple of 32)
    // the block's slices all in one segment (always for one system): bucket maxima in shared memory too
    const int64_t rb = (int64_t)blockIdx.x * blockDim.x;
    const int64_t re = (rb + blockDim.x < rows ? rb + blockDim.x : rows) - 1;
    const int sg0 = seg_of(slice_seg, rb >> 5);
    const bool one_seg = seg_of(slice_seg, re >> 5) == sg0;
    if (threadIdx.x < 8) {
        s_cnt[threadIdx.x] = 0;
        s_wmax[threadIdx.x] = 0;
        s_wmin[threadIdx.x] = 0x7fffffff;
        reinterpret_cast<VT*>(s_bmax)[threadIdx.x] = VT(0);
    }
    if (threadIdx.x == 0) s_dmax = 0;
    __syncthreads();
    if (live) classify_rows(r, n, nslices, sptr, col, val, rowlen, P, thr_g, id, widths, colmax, slice_seg, packed,
                            bmax, one_seg, s_cnt, s_wmax, s_wmin, reinterpret_cast<VT*>(s_bmax), &s_dmax);
    __syncthreads();
    if ((int)threadIdx.x < P.q) {
        const int k = threadIdx.x;
        if (s_cnt[k]) atomicAdd(nnzk + k, s_cnt[k]);
        if (s_wmax[k]) atomicMax(wmax + k, s_wmax[k]);
        atomicMin(wmin + k, s_wmin[k]);
        const VT m = reinterpret_cast<VT*>(s_bmax)[k];
        if (one_seg && m > VT(0)) atomic_max_nonneg(bmax + sg0 * 8 + k, m);
    }
    if (threadIdx.x == 0 && s_dmax) atomicMax(dmax, s_dmax);
}

// least power of two s = 2^e with maxabs <= fmax * 2^e (1 if maxabs == 0)
__device__ __forceinline__ float pow2_scale(double maxabs, double fmax) {
    if (!(maxabs > 0.0)) return 1.0f;
    // both normal: maxabs = ma 2^Ea, fmax = mf 2^Ef with ma, mf in [1, 2), so
    // e = Ea - Ef when ma <= mf and Ea - Ef + 1 otherwise (integer fields only)
    const long long ab = __double_as_longlong(maxabs), fb = __double_as_longlong(fmax);
    const int Ea = (int)((ab >> 52) & 0x7ff), Ef = (int)((fb >> 52) & 0x7ff);
    if (Ea > 0 && Ea < 0x7ff && Ef > 0 && Ef < 0x7ff) {
        const long long m = 0xfffffffffffffLL;
        const int e = Ea - Ef + ((ab & m) > (fb & m) ? 1 : 0);
        if (e >= -126 && e <= 127) return __int_as_float((e + 127) << 23);
    }
    int E;
    frexp(maxabs / fmax, &E);
    int e = E - 2;
    while (maxabs > ldexp(fmax, e)) ++e;
    while (e > -1074 && maxabs <= ldexp(fmax, e - 1)) --e;
    return (float)ldexp(1.0, e);
}

template <typename VT>
__global__ void k_bucket_scales(const __grid_constant__ BucketParams P, int nseg, const VT* __restrict__ bmax,
                                float* __restrict__ scale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = i & 7;
    if (i >= nseg * 8 || k >= P.q) return;
    scale[i] = P.precs[k] == BSPAI_FP16 ? pow2_scale((double)bmax[i], 65504.0) : 1.0f;
}

// per-slice copy of an fp16 bucket's scale (batches of several systems)
__global__ void k_slice_scales(int nslices, const int32_t* __restrict__ slice_seg, const float* __restrict__ scale,
                               int k, float* __restrict__ out) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nslices) out[s] = scale[slice_seg[s] * 8 + k];
}

template <typename VT>
__global__ void k_col_scales(int n, const VT* __restrict__ colmax, float* __restrict__ colscale) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) colscale[j] = pow2_scale((double)colmax[j], 448.0);
}

__device__ __forceinline__ void store_val(void* dst, int64_t p, int prec, float m, float scale, float cs) {
    switch (prec) {
    case BSPAI_FP64: reinterpret_cast<double*>(dst)[p] = (double)m; break;
    case BSPAI_FP32: reinterpret_cast<float*>(dst)[p] = m; break;
    case BSPAI_FP16: reinterpret_cast<__half*>(dst)[p] = __float2half_rn(__fdiv_rn(m, scale)); break;
    case BSPAI_BF16: reinterpret_cast<__nv_bfloat16*>(dst)[p] = __float2bfloat16_rn(m); break;
    case BSPAI_E4M3:
        reinterpret_cast<__nv_fp8_storage_t*>(dst)[p] =
            __nv_cvt_float_to_fp8(__fdiv_rn(m, cs), __NV_SATFINITE, __NV_E4M3);
        break;
    default: break;
    }
}

// the same from an fp64 value (bucketing A): one rounding from fp64 to the format
__device__ __forceinline__ void store_val(void* dst, int64_t p, int prec, double m, float scale, float cs) {
    switch (prec) {
    case BSPAI_FP64: reinterpret_cast<double*>(dst)[p] = m; break;
    case BSPAI_FP32: reinterpret_cast<float*>(dst)[p] = __double2float_rn(m); break;
    case BSPAI_FP16: reinterpret_cast<__half*>(dst)[p] = __double2half(__ddiv_rn(m, (double)scale)); break;
    case BSPAI_BF16: reinterpret_cast<__nv_bfloat16*>(dst)[p] = __double2bfloat16(m); break;
    case BSPAI_E4M3:
        reinterpret_cast<__nv_fp8_storage_t*>(dst)[p] =
            __nv_cvt_double_to_fp8(__ddiv_rn(m, (double)cs), __NV_SATFINITE, __NV_E4M3);
        break;
    default: break;
    }
}

__device__ __forceinline__ void store_zero(void* dst, int64_t p, int prec) {
    switch (prec) {
    case BSPAI_FP64: reinterpret_cast<double*>(dst)[p] = 0.0; break;
    case BSPAI_FP32: reinterpret_cast<float*>(dst)[p] = 0.0f; break;
    case BSPAI_FP16: reinterpret_cast<__half*>(dst)[p] = __float2half_rn(0.0f); break;
    case BSPAI_BF16: reinterpret_cast<__nv_bfloat16*>(dst)[p] = __float2bfloat16_rn(0.0f); break;
    case BSPAI_E4M3: reinterpret_cast<__nv_fp8_storage_t*>(dst)[p] = 0; break;
    default: break;
    }
}

template <typename VT>
__global__ void __launch_bounds__(256) k_pack(int n, int nslices, const int64_t* __restrict__ sptr,
                                              const int32_t* __restrict__ col, const VT* __restrict__ val,
                                              const int32_t* __restrict__ rowlen, const int8_t* __restrict__ id,
                                              const __grid_constant__ PackDst D, const float* __restrict__ scale_g,
                                              const float* __restrict__ colscale,
                                              const int32_t* __restrict__ slice_seg) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (int64_t)nslices * kSlice) return;
    const int64_t s = r >> 5;
    const int lane = (int)(r & 31);
    const float* scale = scale_g + seg_of(slice_seg, s) * 8;
    int cnt[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) cnt[k] = 0;
    if (r < n) {
        const int64_t b = sptr[s] + lane;
        const int len = rowlen[r];
        for (int l = 0; l < len; ++l) {
            const int64_t slot = b + (int64_t)l * kSlice;
            const int k = id[slot];
            int pos = 0;
#pragma unroll
            for (int kk = 0; kk < 8; ++kk)
                if (kk == k) pos = cnt[kk]++;
            if (D.precs[k] == BSPAI_DROP) continue;
            const int c = col[slot];
            const int64_t dst = sell_slot(D.sptr[k][s], lane, pos, D.packed);
            if (D.col16[k]) D.col16[k][dst] = (int16_t)(c - r);
            else D.col[k][dst] = c;
            store_val(D.val[k], dst, D.precs[k], val[slot], scale[k], colscale ? colscale[c] : 1.0f);
        }
    }
    for (int k = 0; k < D.q; ++k) {
        if (D.precs[k] == BSPAI_DROP) continue;
        const int width = (int)((D.sptr[k][s + 1] - D.sptr[k][s]) / kSlice);
        int c0 = 0;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
            if (kk == k) c0 = cnt[kk];
        for (int l = c0; l < width; ++l) {
            const int64_t dst = sell_slot(D.sptr[k][s], lane, l, D.packed);
            if (D.col16[k]) D.col16[k][dst] = kCol16Pad;
            else D.col[k][dst] = -1;
            store_zero(D.val[k], dst, D.precs[k]);
        }
    }
}

// per nonzero in CSR order: bucket id and the value the product uses
__global__ void k_bucket_export(int n, const int64_t* __restrict__ msptr, const int32_t* __restrict__ mrowlen,
                                const int32_t* __restrict__ mcsr, const int8_t* __restrict__ id_sell,
                                const __grid_constant__ BMDev B, int8_t* __restrict__ ids,
                                double* __restrict__ stored) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t s = r >> 5;
    const int lane = (int)(r & 31);
    const int64_t b = msptr[s] + lane;
    const int len = mrowlen[r];
    const int o = mcsr[r];
    int cnt[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) cnt[k] = 0;
    for (int l = 0; l < len; ++l) {
        const int k = id_sell[b + (int64_t)l * kSlice];
        int pos = 0;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
            if (kk == k) pos = cnt[kk]++;
        if (ids) ids[o + l] = (int8_t)k;
        if (!stored) continue;
        const BucketDev& D = B.b[k];
        double v = 0.0;
        if (D.prec != BSPAI_DROP) {
            const int64_t p = sell_slot(D.sptr[s], lane, pos, D.packed);
            const int c = sell_col(D.col, D.col16, p, r);
            switch (D.prec) {
            case BSPAI_FP64: v = reinterpret_cast<const double*>(D.val)[p]; break;
            case BSPAI_FP32: v = reinterpret_cast<const float*>(D.val)[p]; break;
            case BSPAI_FP16:
                v = (double)__half2float(reinterpret_cast<const __half*>(D.val)[p]) *
                    (D.slicescale ? D.slicescale[s] : D.scale);
                break;
            case BSPAI_BF16: v = (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(D.val)[p]); break;
            case BSPAI_E4M3: {
                __nv_fp8_e4m3 e;
                e.__x = reinterpret_cast<const __nv_fp8_storage_t*>(D.val)[p];
                v = (double)float(e) * D.colscale[c];
                break;
            }
            default: break;
            }
        }
        stored[o + l] = v;
    }
}

}  // namespace bspai

using namespace bspai;

// The matrix a bucketing reads: SELL structure, values (fp32 for M, fp64 for
// A), row lengths and CSR row pointers (for export in CSR order).
template <typename VT>
struct BucketSrc {
    int n;
    int64_t nnz;
    const Sell* sell;
    const VT* val;
    const int32_t* rowlen;
    const int32_t* csr_row_ptr;
};

// Bucketing of one system (slice_seg = null, nseg = 1) or of nseg independent
// systems stacked block-diagonally (slice_seg: system of every 32-row slice).
template <typename VT>
static int bucket_impl(const BucketSrc<VT>& S, double bucket_eps, const int32_t* precs, int32_t q,
                       const int32_t* slice_seg, int nseg, cudaStream_t s, bspai_BM_h* out,
                       bspai_bucket_info_t* info) {
    if (!out) return set_error(BSPAI_ERR_INVALID, "bspai_bucket: null out");
    *out = nullptr;
    if (!precs || q < 1 || q > 8) return set_error(BSPAI_ERR_INVALID, "bspai_bucket: need 1 <= q <= 8 precisions");
    if (!(bucket_eps > 0.0)) return set_error(BSPAI_ERR_INVALID, "bspai_bucket: bucket_eps must be > 0");
    BucketParams P{};
    P.q = q;
    P.eps = bucket_eps;
    int n_e4m3 = 0;
    for (int k = 0; k < q; ++k) {
        P.precs[k] = precs[k];
        P.uk[k] = unit_roundoff(precs[k]);
        if (P.uk[k] < 0) return set_error(BSPAI_ERR_INVALID, "bspai_bucket: precision %d not a storage format", precs[k]);
        if (k > 0 && !(P.uk[k] > P.uk[k - 1]))
            return set_error(BSPAI_ERR_INVALID, "bspai_bucket: precisions must have increasing unit roundoff");
        n_e4m3 += precs[k] == BSPAI_E4M3;
    }
    if (n_e4m3 > 1) return set_error(BSPAI_ERR_UNSUPPORTED, "bspai_bucket: at most one e4m3 bucket");
    const int n = S.n;
    const int nsl = S.sell->nslices;
    auto* B = new bspai_bucketed();
    B->magic = kMagicBM;
    B->stream = s;
    B->n = n;
    B->nnz = S.nnz;
    B->q = q;
    for (int k = 0; k < q; ++k) B->precs[k] = precs[k];

    // scratch: norm, thresholds, widths, counts, maxima
    double* d_norm = nullptr;
    double* d_thr = nullptr;
    int64_t* d_w = nullptr;
    unsigned long long* d_nnzk = nullptr;
    VT* d_bmax = nullptr;
    float* d_scale = nullptr;
    VT* d_colmax = nullptr;
    int* d_wmax = nullptr;
    unsigned* d_dmax = nullptr;
    int* d_wmin = nullptr;
    auto cleanup = [&]() {
        dfree(d_norm, s); dfree(d_thr, s); dfree(d_w, s); dfree(d_nnzk, s);
        dfree(d_bmax, s); dfree(d_scale, s); dfree(d_colmax, s); dfree(d_wmax, s); dfree(d_dmax, s);
        dfree(d_wmin, s);
    };
    // One system: the packed slot arrangement, with 16-bit column differences
    // when every |c - r| fits (the SpMV reads a row's slots four at a time).
    // A batch keeps the plain arrangement its batched solver reads.
    const int packed = slice_seg ? 0 : 1;
    auto fail = [&](int code) {
        cleanup();
        bspai_free(B);
        return code;
    };
    int rc;
    ProfScope ps(BSPAI_K_BUCKET, s);
    // private copy of M's structure (for export) and the bucket id per slot
    B->msell.n = n;
    B->msell.nslices = nsl;
    B->msell.slots = S.sell->slots;
    if ((rc = dalloc_t(&B->msell.sptr, (size_t)nsl + 1, s))) return fail(rc);
    if ((rc = dalloc_t(&B->msell.col, (size_t)S.sell->slots, s))) return fail(rc);
    if ((rc = dalloc_t(&B->mrowlen, (size_t)n, s))) return fail(rc);
    if ((rc = dalloc_t(&B->mcsr_row_ptr, (size_t)n + 1, s))) return fail(rc);
    if ((rc = dalloc_t(&B->id_sell, (size_t)S.sell->slots, s))) return fail(rc);
    if ((rc = dalloc_t(&d_norm, (size_t)nseg, s))) return fail(rc);
    if ((rc = dalloc_t(&d_thr, (size_t)nseg * 8, s))) return fail(rc);
    if ((rc = dalloc_t(&d_w, (size_t)q * (nsl + 1), s))) return fail(rc);
    if ((rc = dalloc_t(&d_nnzk, 8, s))) return fail(rc);
    if ((rc = dalloc_t(&d_bmax, (size_t)nseg * 8, s))) return fail(rc);
    if ((rc = dalloc_t(&d_scale, (size_t)nseg * 8, s))) return fail(rc);
    if ((rc = dalloc_t(&d_wmax, 8, s))) return fail(rc);
    if ((rc = dalloc_t(&d_dmax, 1, s))) return fail(rc);
    if ((rc = dalloc_t(&d_wmin, 8, s))) return fail(rc);
    if (n_e4m3) {
        if ((rc = dalloc_t(&d_colmax, (size_t)n, s))) return fail(rc);
        if ((rc = dalloc_t(&B->colscale, (size_t)n, s))) return fail(rc);
    }
    cudaError_t e = cudaSuccess;
    e = cudaMemcpyAsync(B->msell.sptr, S.sell->sptr, sizeof(int64_t) * ((size_t)nsl + 1), cudaMemcpyDeviceToDevice, s);
    if (!e) e = cudaMemcpyAsync(B->msell.col, S.sell->col, sizeof(int32_t) * (size_t)S.sell->slots, cudaMemcpyDeviceToDevice, s);
    if (!e) e = cudaMemcpyAsync(B->mrowlen, S.rowlen, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
    if (!e) e = cudaMemcpyAsync(B->mcsr_row_ptr, S.csr_row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, s);
    if (!e) e = cudaMemsetAsync(d_norm, 0, sizeof(double) * (size_t)nseg, s);
    if (!e) e = cudaMemsetAsync(d_nnzk, 0, 8 * sizeof(unsigned long long), s);
    if (!e) e = cudaMemsetAsync(d_bmax, 0, 8 * sizeof(VT) * (size_t)nseg, s);
    if (!e) e = cudaMemsetAsync(d_wmax, 0, 8 * sizeof(int), s);
    if (!e) e = cudaMemsetAsync(d_dmax, 0, sizeof(unsigned), s);
    if (!e) e = cudaMemsetAsync(d_wmin, 0x7f, 8 * sizeof(int), s);  // 0x7f7f7f7f: above any width
    if (!e) e = cudaMemsetAsync(d_w, 0, sizeof(int64_t) * (size_t)q * (nsl + 1), s);
    if (!e && d_colmax) e = cudaMemsetAsync(d_colmax, 0, sizeof(VT) * (size_t)n, s);
    if (e) return fail(cuda_error(e, "bspai_bucket setup", __FILE__, __LINE__));
    const unsigned g_rows = (unsigned)ceil_div((int64_t)nsl * kSlice, 256);
    const unsigned g_seg = (unsigned)ceil_div(nseg, 256), g_seg8 = (unsigned)ceil_div((int64_t)nseg * 8, 256);
    if (n > 0) {
        k_norm_rows<VT><<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, S.sell->sptr, S.val, S.rowlen, slice_seg, d_norm);
        note_launch();
        k_thresholds<<<g_seg, 256, 0, s>>>(P, nseg, d_norm, d_thr);
        note_launch();
        k_classify<VT><<<g_rows, 256, 0, s>>>(n, nsl, S.sell->sptr, S.sell->col, S.val, S.rowlen, P, d_thr,
                                              B->id_sell, d_w, d_nnzk, d_bmax, d_colmax, d_wmax, slice_seg,
                                              packed, d_dmax, d_wmin);
        note_launch();
        k_bucket_scales<VT><<<g_seg8, 256, 0, s>>>(P, nseg, d_bmax, d_scale);
        note_launch();
        if (d_colmax) {
            k_col_scales<VT><<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, d_colmax, B->colscale);
            note_launch();
        }
    } else {
        k_thresholds<<<g_seg, 256, 0, s>>>(P, nseg, d_norm, d_thr);
        note_launch();
        k_bucket_scales<VT><<<g_seg8, 256, 0, s>>>(P, nseg, d_bmax, d_scale);
        note_launch();
    }
    if ((e = cudaGetLastError())) return fail(cuda_error(e, "bucket classify", __FILE__, __LINE__));
    for (int k = 0; k < q; ++k) {
        B->b[k].n = n;
        B->b[k].nslices = nsl;
        if ((rc = dalloc_t(&B->b[k].sptr, (size_t)nsl + 1, s))) return fail(rc);
        if ((rc = scan_exclusive_i64(d_w + (size_t)k * (nsl + 1), B->b[k].sptr, nsl, s))) return fail(rc);
    }
    // sizes back to the host
    int64_t slots[8] = {0};
    unsigned long long nnzk[8] = {0};
    double hthr[8] = {0};
    std::vector<double> hnorms((size_t)nseg, 0.0);
    float hscale[8] = {0};
    int hwmax[8] = {0};
    unsigned hdmax = 0;
    int hwmin[8] = {0};
    for (int k = 0; k < q; ++k)
        if ((e = cudaMemcpyAsync(&slots[k], B->b[k].sptr + nsl, sizeof(int64_t), cudaMemcpyDeviceToHost, s)))
            return fail(cuda_error(e, "bucket sizes", __FILE__, __LINE__));
    e = cudaMemcpyAsync(nnzk, d_nnzk, sizeof nnzk, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(hthr, d_thr, sizeof hthr, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(hnorms.data(), d_norm, sizeof(double) * (size_t)nseg, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(hscale, d_scale, sizeof hscale, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(hwmax, d_wmax, sizeof hwmax, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(&hdmax, d_dmax, sizeof hdmax, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(hwmin, d_wmin, sizeof hwmin, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return fail(cuda_error(e, "bucket sizes", __FILE__, __LINE__));
    double hnorm = 0.0;
    for (double v : hnorms) hnorm = v > hnorm ? v : hnorm;
    PackDst D{};
    D.q = q;
    D.packed = packed;
    const bool idx16 = packed && hdmax <= 32767u;
    int64_t bytes = 0;
    for (int k = 0; k < q; ++k) {
        B->nnz_k[k] = (int64_t)nnzk[k];
        B->scale[k] = hscale[k];
        B->maxw[k] = hwmax[k];
        B->b[k].maxw = hwmax[k];
        B->b[k].packed = packed;
        // every slice equally wide (a stencil's buckets): slice starts need no table
        B->b[k].ellw = (packed && nsl > 0 && hwmin[k] == hwmax[k] && hwmax[k] > 0) ? hwmax[k] : 0;
        D.precs[k] = precs[k];
        D.sptr[k] = B->b[k].sptr;
        D.scale[k] = hscale[k];
        bytes += (int64_t)sizeof(int64_t) * (nsl + 1);
        if (precs[k] == BSPAI_DROP) {
            B->b[k].slots = 0;
            continue;
        }
        B->b[k].slots = slots[k];
        if (idx16) {
            if ((rc = dalloc_t(&B->b[k].col16, (size_t)slots[k], s))) return fail(rc);
        } else {
            if ((rc = dalloc_t(&B->b[k].col, (size_t)slots[k], s))) return fail(rc);
        }
        if ((rc = dalloc(&B->val[k], (size_t)slots[k] * prec_bytes(precs[k]), s))) return fail(rc);
        D.col[k] = B->b[k].col;
        D.col16[k] = B->b[k].col16;
        D.val[k] = B->val[k];
        bytes += slots[k] * (int64_t)((idx16 ? 2 : 4) + prec_bytes(precs[k]));
    }
    if (B->colscale) bytes += (int64_t)sizeof(float) * n;
    if (n > 0) {
        k_pack<VT><<<g_rows, 256, 0, s>>>(n, nsl, S.sell->sptr, S.sell->col, S.val, S.rowlen, B->id_sell, D, d_scale,
                                          B->colscale, slice_seg);
        note_launch();
        if ((e = cudaGetLastError())) return fail(cuda_error(e, "k_pack", __FILE__, __LINE__));
    }
    if (slice_seg && nsl > 0) {
        // each system's fp16 scale, per 32-row slice, for the SpMV kernels
        for (int k = 0; k < q; ++k) {
            if (precs[k] != BSPAI_FP16) continue;
            if ((rc = dalloc_t(&B->sscale[k], (size_t)nsl, s))) return fail(rc);
            k_slice_scales<<<(unsigned)ceil_div(nsl, 256), 256, 0, s>>>(nsl, slice_seg, d_scale, k, B->sscale[k]);
            note_launch();
            bytes += (int64_t)sizeof(float) * nsl;
        }
        if ((e = cudaGetLastError())) return fail(cuda_error(e, "k_slice_scales", __FILE__, __LINE__));
    }
    cleanup();
    if (info) {
        info->q = q;
        double num = 0, num8 = 0, tot = 0;
        for (int k = 0; k < 8; ++k) {
            info->precs[k] = k < q ? precs[k] : -1;
            info->nnz_k[k] = k < q ? B->nnz_k[k] : 0;
            info->slots_k[k] = k < q ? B->b[k].slots : 0;
            info->thresholds[k] = k < q ? hthr[k] : 0.0;
        }
        for (int k = 0; k < q; ++k) {
            int bits = prec_bits(precs[k]);
            int bits8 = (k == q - 1 && precs[k] == BSPAI_DROP) ? 8 : bits;
            num += (double)B->nnz_k[k] * bits;
            num8 += (double)B->nnz_k[k] * bits8;
            tot += (double)B->nnz_k[k];
        }
        double den = tot * prec_bits(precs[0]);
        info->norm_inf = hnorm;
        info->storage_pct = den > 0 ? 100.0 * num / den : 0.0;
        info->storage_pct_last8 = den > 0 ? 100.0 * num8 / den : 0.0;
        info->bytes = bytes;
        e = cudaStreamSynchronize(s);
        if (e) {
            int code = cuda_error(e, "bspai_bucket", __FILE__, __LINE__);
            bspai_free(B);
            return code;
        }
    }
    *out = B;
    return BSPAI_OK;
}

// system of every 32-row slice from the system row offsets (multiples of 32)
__global__ void k_slice_seg(int nseg, const int32_t* __restrict__ row_off, int32_t* __restrict__ slice_seg,
                            int* __restrict__ bad) {
    const int sg = blockIdx.x * blockDim.x + threadIdx.x;
    if (sg >= nseg) return;
    const int a = row_off[sg], b = row_off[sg + 1];
    if ((a & 31) || (b & 31) || b < a) {
        atomicOr(bad, 1);
        return;
    }
    for (int s = a >> 5; s < (b >> 5); ++s) slice_seg[s] = sg;
}

extern "C" {

static BucketSrc<float> m_source(const bspai_spai* M) {
    return BucketSrc<float>{M->n, M->nnz, &M->sell, M->val, M->rowlen, M->csr_row_ptr};
}

int bspai_bucket(bspai_M_h M, double bucket_eps, const int32_t* precs, int32_t q, bspai_stream_t st,
                 bspai_BM_h* out, bspai_bucket_info_t* info) {
    if (out) *out = nullptr;
    if (!M || M->magic != kMagicM) return set_error(BSPAI_ERR_INVALID, "bspai_bucket: bad M handle");
    return bucket_impl(m_source(M), bucket_eps, precs, q, nullptr, 1, (cudaStream_t)st, out, info);
}

int bspai_bucket_A(bspai_A_h A, double bucket_eps, const int32_t* precs, int32_t q, bspai_stream_t st,
                   bspai_BM_h* out, bspai_bucket_info_t* info) {
    if (out) *out = nullptr;
    if (!A || A->magic != kMagicA) return set_error(BSPAI_ERR_INVALID, "bspai_bucket_A: bad A handle");
    if (!A->rowlen || !A->csr_row_ptr)
        return set_error(BSPAI_ERR_UNSUPPORTED, "bspai_bucket_A: A has no row lengths (a transposed A)");
    const BucketSrc<double> src{A->n, A->nnz, &A->sell, A->val64, A->rowlen, A->csr_row_ptr};
    return bucket_impl(src, bucket_eps, precs, q, nullptr, 1, (cudaStream_t)st, out, info);
}

int bspai_bucket_batched(bspai_M_h M, const int32_t* row_off, int32_t nsys, double bucket_eps, const int32_t* precs,
                         int32_t q, bspai_stream_t st, bspai_BM_h* out, bspai_bucket_info_t* info) {
    cudaStream_t s = (cudaStream_t)st;
    if (!out) return set_error(BSPAI_ERR_INVALID, "bspai_bucket_batched: null out");
    *out = nullptr;
    if (!M || M->magic != kMagicM) return set_error(BSPAI_ERR_INVALID, "bspai_bucket_batched: bad M handle");
    if (!row_off || nsys < 1) return set_error(BSPAI_ERR_INVALID, "bspai_bucket_batched: need nsys >= 1 offsets");
    int last = -1, first = -1;
    CUDA_TRY(cudaMemcpyAsync(&first, row_off, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(&last, row_off + nsys, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (first != 0 || last != M->n)
        return set_error(BSPAI_ERR_INVALID, "bspai_bucket_batched: row_off must run from 0 to n = %d", M->n);
    const int nsl = M->sell.nslices;
    int32_t* slice_seg = nullptr;
    int* bad = nullptr;
    BSPAI_TRY(dalloc_t(&slice_seg, (size_t)(nsl > 0 ? nsl : 1), s));
    BSPAI_TRY(dalloc_t(&bad, 1, s));
    CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
    CUDA_TRY(cudaMemsetAsync(slice_seg, 0, sizeof(int32_t) * (size_t)(nsl > 0 ? nsl : 1), s));
    k_slice_seg<<<(unsigned)ceil_div(nsys, 256), 256, 0, s>>>(nsys, row_off, slice_seg, bad);
    note_launch();
    CUDA_LAUNCH_CHECK();
    int hbad = 0;
    CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    int rc;
    if (hbad)
        rc = set_error(BSPAI_ERR_INVALID, "bspai_bucket_batched: system offsets must be non-decreasing multiples of 32");
    else
        rc = bucket_impl(m_source(M), bucket_eps, precs, q, slice_seg, nsys, s, out, info);
    dfree(slice_seg, s);
    dfree(bad, s);
    return rc;
}

int bspai_bucket_export(bspai_BM_h BM, int8_t* ids, double* stored, bspai_stream_t st) {
    cudaStream_t s = (cudaStream_t)st;
    if (!BM || BM->magic != kMagicBM) return set_error(BSPAI_ERR_INVALID, "bspai_bucket_export: bad handle");
    if (!BM->msell.sptr)
        return set_error(BSPAI_ERR_UNSUPPORTED, "bspai_bucket_export: not available for a transposed bucketed M");
    if (BM->n == 0 || (!ids && !stored)) return BSPAI_OK;
    k_bucket_export<<<(unsigned)ceil_div(BM->n, 256), 256, 0, s>>>(BM->n, BM->msell.sptr, BM->mrowlen,
                                                                   BM->mcsr_row_ptr, BM->id_sell, BM->dev(), ids,
                                                                   stored);
    note_launch();
    CUDA_LAUNCH_CHECK();
    return BSPAI_OK;
}

}  // extern "C"
