// spmv_row.cuh -- per-row pieces of the adaptive-precision SpMV (Alg 2.3),
// shared by the SpMV kernels and the batched GMRES kernel so that every
// product on the path uses the same operations in the same order.
#pragma once

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

// an entry of x: through the read-only path, or (CG) from L2 -- for a vector
// that other blocks of the same launch write (the batched solver's teams)
template <bool CG, typename XT>
__device__ __forceinline__ XT ldx(const XT* p) {
    if constexpr (CG) return __ldcg(p);
    else return __ldg(p);
}

// column of slot p of row r, read through the read-only path
__device__ __forceinline__ int sell_col_ldg(const BucketDev& B, int64_t p, int64_t r) {
    if (B.col16) {
        const int d = __ldg(B.col16 + p);
        return d == kCol16Pad ? -1 : (int)(r + d);
    }
    return __ldg(B.col + p);
}

// fp32 partial sum of one row over one narrow bucket (w slots per row of its
// slice starting at sbase, either slot arrangement).  Loads are issued four
// slots ahead of the (strictly sequential) accumulation.
template <int PREC, typename XT, bool CG = false>
__device__ __forceinline__ float row_partial_f32(const BucketDev& B, int64_t sbase, int w,
                                                 const XT* __restrict__ x, int64_t r) {
    // e4m3 scales: per column of M, or per row of a transposed M; fp16: per bucket or per slice
    const float* st = B.colscale ? B.colscale : B.rowscale;
    const float sc = B.slicescale ? __ldg(B.slicescale + (r >> 5)) : B.scale;
    const int lane = (int)(r & 31);
    float acc = 0.0f;
    int l = 0;
    for (; l + 3 < w; l += 4) {
        int64_t p[4];
        int c[4];
        float v[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            p[u] = sell_slot(sbase, lane, l + u, B.packed);
            c[u] = sell_col_ldg(B, p[u], r);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (c[u] >= 0) {
                v[u] = decode<PREC>(B.val, p[u], sc, st, B.colscale ? c[u] : (int)r);
                xv[u] = to_f32<XT>(ldx<CG>(x + c[u]));
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (c[u] >= 0) acc = __fadd_rn(acc, __fmul_rn(v[u], xv[u]));
    }
    for (; l < w; ++l) {
        const int64_t p = sell_slot(sbase, lane, l, B.packed);
        const int c = sell_col_ldg(B, p, r);
        if (c >= 0) {
            const float v = decode<PREC>(B.val, p, sc, st, B.colscale ? c : (int)r);
            acc = __fadd_rn(acc, __fmul_rn(v, to_f32<XT>(ldx<CG>(x + c))));
        }
    }
    return acc;
}

template <typename XT, bool CG = false>
__device__ __forceinline__ double row_partial_f64(const BucketDev& B, int64_t sbase, int w,
                                                  const XT* __restrict__ x, int64_t r) {
    const double* val = reinterpret_cast<const double*>(B.val);
    const int lane = (int)(r & 31);
    double acc = 0.0;
    int l = 0;
    for (; l + 3 < w; l += 4) {
        int64_t p[4];
        int c[4];
        double v[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            p[u] = sell_slot(sbase, lane, l + u, B.packed);
            c[u] = sell_col_ldg(B, p[u], r);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (c[u] >= 0) {
                v[u] = __ldg(val + p[u]);
                xv[u] = (double)ldx<CG>(x + c[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (c[u] >= 0) acc = __dadd_rn(acc, __dmul_rn(v[u], xv[u]));
    }
    for (; l < w; ++l) {
        const int64_t p = sell_slot(sbase, lane, l, B.packed);
        const int c = sell_col_ldg(B, p, r);
        if (c >= 0) acc = __dadd_rn(acc, __dmul_rn(__ldg(val + p), (double)ldx<CG>(x + c)));
    }
    return acc;
}

// one narrow-bucket value to fp32, format chosen at run time (uniform per warp)
__device__ __forceinline__ float decode_rt(const BucketDev& B, int64_t p, int c, int64_t r) {
    switch (B.prec) {
    case BSPAI_FP32: return decode<BSPAI_FP32>(B.val, p, B.scale, nullptr, c);
    case BSPAI_FP16:
        return decode<BSPAI_FP16>(B.val, p, B.slicescale ? __ldg(B.slicescale + (r >> 5)) : B.scale, nullptr, c);
    case BSPAI_BF16: return decode<BSPAI_BF16>(B.val, p, B.scale, nullptr, c);
    default:
        return B.colscale ? decode<BSPAI_E4M3>(B.val, p, B.scale, B.colscale, c)
                          : decode<BSPAI_E4M3>(B.val, p, B.scale, B.rowscale, (int)r);
    }
}

// y_i = sum_k y_i^(k) for row r of a bucketed matrix: each bucket's partial sum
// in ascending column order (fp64 for an fp64 bucket, fp32 otherwise), the
// partial sums added in fp64 in bucket order.
template <typename XT, bool CG = false>
__device__ __forceinline__ double bucketed_row(const BMDev& M, int64_t r, const XT* __restrict__ x) {
    const int64_t s = r >> 5;
    double yi = 0.0;
    for (int k = 0; k < M.q; ++k) {
        const BucketDev& B = M.b[k];
        if (B.prec == BSPAI_DROP) continue;  // dropped entries are not stored
        const int64_t sb = B.sptr[s];
        const int w = (int)((B.sptr[s + 1] - sb) >> 5);
        switch (B.prec) {
        case BSPAI_FP64: yi = __dadd_rn(yi, row_partial_f64<XT, CG>(B, sb, w, x, r)); break;
        case BSPAI_FP32: yi = __dadd_rn(yi, (double)row_partial_f32<BSPAI_FP32, XT, CG>(B, sb, w, x, r)); break;
        case BSPAI_FP16: yi = __dadd_rn(yi, (double)row_partial_f32<BSPAI_FP16, XT, CG>(B, sb, w, x, r)); break;
        case BSPAI_BF16: yi = __dadd_rn(yi, (double)row_partial_f32<BSPAI_BF16, XT, CG>(B, sb, w, x, r)); break;
        case BSPAI_E4M3: yi = __dadd_rn(yi, (double)row_partial_f32<BSPAI_E4M3, XT, CG>(B, sb, w, x, r)); break;
        default: break;
        }
    }
    return yi;
}

// Two rows at once (rows ra and rb, in slices of their own): the same partial
// sums as row_partial_f32 / row_partial_f64 for each row, in the same order,
// with the loads of both rows issued together so that each thread keeps two
// independent chains of gathers in flight.  Plain slot arrangement and int32
// columns only: the batched bucketing, whose solver uses these, keeps them.
template <int PREC, typename XT, bool CG = false>
__device__ __forceinline__ void row_partial2_f32(const BucketDev& B, int64_t pa, int64_t ea, int64_t pb, int64_t eb,
                                                 const XT* __restrict__ x, int64_t ra, int64_t rb, float& acc_a,
                                                 float& acc_b) {
    const float* st = B.colscale ? B.colscale : B.rowscale;
    const float sca = B.slicescale ? __ldg(B.slicescale + (ra >> 5)) : B.scale;
    const float scb = B.slicescale ? __ldg(B.slicescale + (rb >> 5)) : B.scale;
    float aa = 0.0f, ab = 0.0f;
    for (; pa < ea || pb < eb; pa += 64, pb += 64) {
        int c[4];
        c[0] = pa < ea ? __ldg(B.col + pa) : -1;
        c[1] = pa + 32 < ea ? __ldg(B.col + pa + 32) : -1;
        c[2] = pb < eb ? __ldg(B.col + pb) : -1;
        c[3] = pb + 32 < eb ? __ldg(B.col + pb + 32) : -1;
        float v[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (c[u] >= 0) {
                const int64_t p = u < 2 ? pa + 32 * u : pb + 32 * (u - 2);
                const int64_t r = u < 2 ? ra : rb;
                v[u] = decode<PREC>(B.val, p, u < 2 ? sca : scb, st, B.colscale ? c[u] : (int)r);
                xv[u] = to_f32<XT>(ldx<CG>(x + c[u]));
            }
        }
        if (c[0] >= 0) aa = __fadd_rn(aa, __fmul_rn(v[0], xv[0]));
        if (c[1] >= 0) aa = __fadd_rn(aa, __fmul_rn(v[1], xv[1]));
        if (c[2] >= 0) ab = __fadd_rn(ab, __fmul_rn(v[2], xv[2]));
        if (c[3] >= 0) ab = __fadd_rn(ab, __fmul_rn(v[3], xv[3]));
    }
    acc_a = aa;
    acc_b = ab;
}

template <typename XT, bool CG = false>
__device__ __forceinline__ void row_partial2_f64(const BucketDev& B, int64_t pa, int64_t ea, int64_t pb, int64_t eb,
                                                 const XT* __restrict__ x, double& acc_a, double& acc_b) {
    const double* val = reinterpret_cast<const double*>(B.val);
    double aa = 0.0, ab = 0.0;
    for (; pa < ea || pb < eb; pa += 64, pb += 64) {
        int c[4];
        c[0] = pa < ea ? __ldg(B.col + pa) : -1;
        c[1] = pa + 32 < ea ? __ldg(B.col + pa + 32) : -1;
        c[2] = pb < eb ? __ldg(B.col + pb) : -1;
        c[3] = pb + 32 < eb ? __ldg(B.col + pb + 32) : -1;
        double v[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (c[u] >= 0) {
                const int64_t p = u < 2 ? pa + 32 * u : pb + 32 * (u - 2);
                v[u] = __ldg(val + p);
                xv[u] = (double)ldx<CG>(x + c[u]);
            }
        }
        if (c[0] >= 0) aa = __dadd_rn(aa, __dmul_rn(v[0], xv[0]));
        if (c[1] >= 0) aa = __dadd_rn(aa, __dmul_rn(v[1], xv[1]));
        if (c[2] >= 0) ab = __dadd_rn(ab, __dmul_rn(v[2], xv[2]));
        if (c[3] >= 0) ab = __dadd_rn(ab, __dmul_rn(v[3], xv[3]));
    }
    acc_a = aa;
    acc_b = ab;
}

// bucketed_row for two rows at once (the same sums, bucket by bucket in order)
template <typename XT, bool CG = false>
__device__ __forceinline__ void bucketed_row2(const BMDev& M, int64_t ra, int64_t rb, const XT* __restrict__ x,
                                              double& ya, double& yb) {
    const int64_t sa = ra >> 5, sb = rb >> 5;
    const int la = (int)(ra & 31), lb = (int)(rb & 31);
    double ta = 0.0, tb = 0.0;
    for (int k = 0; k < M.q; ++k) {
        const BucketDev& B = M.b[k];
        const int64_t pa = B.sptr[sa] + la, ea = B.sptr[sa + 1];
        const int64_t pb = B.sptr[sb] + lb, eb = B.sptr[sb + 1];
        if (B.prec == BSPAI_FP64) {
            double a, b;
            row_partial2_f64<XT, CG>(B, pa, ea, pb, eb, x, a, b);
            ta = __dadd_rn(ta, a);
            tb = __dadd_rn(tb, b);
            continue;
        }
        float a = 0.0f, b = 0.0f;
        switch (B.prec) {
        case BSPAI_FP32: row_partial2_f32<BSPAI_FP32, XT, CG>(B, pa, ea, pb, eb, x, ra, rb, a, b); break;
        case BSPAI_FP16: row_partial2_f32<BSPAI_FP16, XT, CG>(B, pa, ea, pb, eb, x, ra, rb, a, b); break;
        case BSPAI_BF16: row_partial2_f32<BSPAI_BF16, XT, CG>(B, pa, ea, pb, eb, x, ra, rb, a, b); break;
        case BSPAI_E4M3: row_partial2_f32<BSPAI_E4M3, XT, CG>(B, pa, ea, pb, eb, x, ra, rb, a, b); break;
        default: continue;  // dropped entries are not stored
        }
        ta = __dadd_rn(ta, (double)a);
        tb = __dadd_rn(tb, (double)b);
    }
    ya = ta;
    yb = tb;
}

// Buckets that contribute nothing (dropped, or with no entries) are left out:
// their partial sums are +0 and adding +0 to a sum that is never -0 changes nothing.
inline BMDev compact_buckets(const BMDev& M) {
    BMDev c = M;
    c.q = 0;
    for (int k = 0; k < M.q; ++k)
        if (M.b[k].prec != BSPAI_DROP && M.b[k].nnz != 0) c.b[c.q++] = M.b[k];
    return c;
}

}  // namespace bspai
