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
#include <atomic>
#include <type_traits>
#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"
#include "spmv_row.cuh"
#include "tma.cuh"

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
        base[k] = __ldg(M.b[k].sptr + s);
        w[k] = (int)((__ldg(M.b[k].sptr + s + 1) - base[k]) >> 5);
    }
    int c[Q][W];
#pragma unroll
    for (int k = 0; k < Q; ++k)
#pragma unroll
        for (int l = 0; l < W; ++l) c[k][l] = l < w[k] ? sell_col_ldg(M.b[k], sell_slot(base[k], lane, l, M.b[k].packed), r) : -1;
    float v[Q][W], xf[Q][W];
    double vd[W], xd[W];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
#pragma unroll
        for (int l = 0; l < W; ++l) {
            const int cc = c[k][l];
            if (cc >= 0) {
                if (F64 && k == 0) {
                    vd[l] = __ldg(reinterpret_cast<const double*>(M.b[0].val) + sell_slot(base[0], lane, l, M.b[0].packed));
                    xd[l] = (double)__ldg(x + cc);
                } else {
                    v[k][l] = decode_rt(M.b[k], sell_slot(base[k], lane, l, M.b[k].packed), cc, r);
                    xf[k][l] = to_f32<XT>(__ldg(x + cc));
                }
            }
        }
    }
    // an fp32 result of at most two narrow partials needs no fp64 arithmetic:
    // fl32(fl64(a + b)) = fl32(a + b) (double rounding through 53 >= 2 * 24 + 2
    // bits is innocuous), and fl64(0 + a) = a
    constexpr bool F32OUT = std::is_same<YT, float>::value && !F64 && Q <= 2;
    double yi = 0.0;
    float yf = 0.0f;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const BucketDev& B = M.b[k];
        if (F64 && k == 0) {
            double acc = 0.0;
#pragma unroll
            for (int l = 0; l < W; ++l)
                if (c[k][l] >= 0) acc = __dadd_rn(acc, __dmul_rn(vd[l], xd[l]));
            for (int l = W; l < w[k]; ++l) {
                const int64_t pp = sell_slot(base[k], lane, l, B.packed);
                const int cc = sell_col_ldg(B, pp, r);
                if (cc >= 0)
                    acc = __dadd_rn(acc, __dmul_rn(__ldg(reinterpret_cast<const double*>(B.val) + pp),
                                                   (double)__ldg(x + cc)));
            }
            yi = __dadd_rn(yi, acc);
        } else {
            float acc = 0.0f;
#pragma unroll
            for (int l = 0; l < W; ++l)
                if (c[k][l] >= 0) acc = __fadd_rn(acc, __fmul_rn(v[k][l], xf[k][l]));
            for (int l = W; l < w[k]; ++l) {
                const int64_t pp = sell_slot(base[k], lane, l, B.packed);
                const int cc = sell_col_ldg(B, pp, r);
                if (cc >= 0) acc = __fadd_rn(acc, __fmul_rn(decode_rt(B, pp, cc, r), to_f32<XT>(__ldg(x + cc))));
            }
            if constexpr (F32OUT) yf = k == 0 ? acc : __fadd_rn(yf, acc);
            else yi = __dadd_rn(yi, (double)acc);
        }
    }
    if (r < M.n) {
        if constexpr (F32OUT) y[r] = yf;
        else y[r] = from_f64<YT>(yi);
    }
}

// ---------------------------------------------------------------- TMA-staged form
// The same product again (same operations, same order, same bits), with the
// matrix streamed into shared memory by the bulk-copy (TMA) engine instead of
// through registers.  Each warp owns a contiguous run of slices and a ring of
// NS stages in shared memory; for every slice, one lane posts the slice's
// column indices and values of every bucket (contiguous ranges in SELL-32:
// 128 w bytes of indices, 32 w b_k bytes of values) as cp.async.bulk copies
// completing on the stage's mbarrier, NS slices ahead of the slice it
// computes.  The bytes in flight per SM are then set by the ring size, not by
// registers, which is what an SpMV with 5-9 entries per row needs to keep HBM
// busy.  Only x (and the e4m3 column scales) are gathered with ordinary loads.
struct StageLayout {
    int32_t col_off[8];  // byte offset of bucket k's indices in a stage
    int32_t val_off[8];  // byte offset of bucket k's values in a stage
    int32_t vbytes[8];   // bytes per stored value of bucket k
    int32_t stage_bytes; // bytes per stage (multiple of 16)
    int32_t ns;          // stages per warp
};

// one stored value (in shared memory) of a narrow bucket to fp32: as decode_rt
__device__ __forceinline__ float decode_sm(const BucketDev& B, const unsigned char* v, int i, int c, int64_t r,
                                           float sc) {
    switch (B.prec) {
    case BSPAI_FP32: return reinterpret_cast<const float*>(v)[i];
    case BSPAI_FP16: return __fmul_rn(__half2float(reinterpret_cast<const __half*>(v)[i]), sc);
    case BSPAI_BF16: return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(v)[i]);
    default: {
        __nv_fp8_e4m3 e;
        e.__x = reinterpret_cast<const __nv_fp8_storage_t*>(v)[i];
        return __fmul_rn(float(e), B.colscale ? __ldg(B.colscale + c) : __ldg(B.rowscale + r));
    }
    }
}

constexpr int kStageHeader = 32;  // per stage: the slice's width of every bucket (int32 x 8)

// set when a warp gave up waiting for its copies (never expected: the copies
// depend on nothing but the memory system); read by stage_timeout_take()
__device__ int g_stage_timeout;

// Launch: blockDim = 32 * warps (<= 256), dynamic shared memory =
// warps * NS * (8 + stage_bytes).  Q: buckets (compacted), W: slots per row
// whose loads are all issued before any arithmetic (wider rows continue in a
// plain loop), F64: bucket 0 is the fp64 bucket.
template <typename XT, typename YT, int Q, int W, bool F64>
__global__ void __launch_bounds__(256) k_bspmv_tma(const __grid_constant__ BMDev M, const XT* __restrict__ x,
                                                   YT* __restrict__ y, const int* __restrict__ jd, int64_t ldx,
                                                   int64_t ldy, int yoff, const __grid_constant__ StageLayout L) {
    extern __shared__ __align__(128) unsigned char sm[];
    if (jd) {
        if (jd[1]) return;
        const int64_t j = jd[0];
        x += j * ldx;
        y += (j + yoff) * ldy;
    }
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    const int NS = L.ns;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm) + (int64_t)wib * NS;
    unsigned char* ring = sm + (size_t)nwb * NS * 8 + (size_t)wib * NS * L.stage_bytes;
    const int64_t nsl = ceil_div(M.n, kSlice);
    const int64_t nwarps = (int64_t)gridDim.x * nwb;
    const int64_t gw = (int64_t)blockIdx.x * nwb + wib;
    const int64_t per = ceil_div(nsl, nwarps);
    const int64_t s0 = gw * per;
    const int64_t s1 = s0 + per < nsl ? s0 + per : nsl;
    if (s0 >= s1) return;
    const int cnt = (int)(s1 - s0);
    // slice pointers of the slices being posted: lane l holds sptr_k[s0 + wb + l]
    int64_t sp[Q];
    int wb = 0;
    auto load_window = [&]() {
        const int64_t si = s0 + wb + lane;
#pragma unroll
        for (int k = 0; k < Q; ++k) sp[k] = si <= s1 ? __ldg(M.b[k].sptr + si) : 0;
    };
    // warp-collective: post the copies of slice s0 + p into stage `st`
    auto post = [&](int p, int st) {
        if (p - wb >= 31) {
            wb += 31;
            load_window();
        }
        unsigned char* stage = ring + (size_t)st * L.stage_bytes;
        int64_t b0[Q], len[Q];
        unsigned total = 0;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            b0[k] = __shfl_sync(0xffffffffu, sp[k], p - wb);
            len[k] = __shfl_sync(0xffffffffu, sp[k], p - wb + 1) - b0[k];
            total += (unsigned)(len[k] * (4 + L.vbytes[k]));
        }
        if (lane == 0) {
            int32_t* hdr = reinterpret_cast<int32_t*>(stage);
#pragma unroll
            for (int k = 0; k < Q; ++k) hdr[k] = (int32_t)(len[k] >> 5);
            mbar_arrive_expect(bars + st, total);
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                if (len[k] == 0) continue;
                bulk_g2s(stage + L.col_off[k], M.b[k].col + b0[k], (unsigned)(len[k] * 4), bars + st);
                bulk_g2s(stage + L.val_off[k],
                         reinterpret_cast<const unsigned char*>(M.b[k].val) + b0[k] * L.vbytes[k],
                         (unsigned)(len[k] * L.vbytes[k]), bars + st);
            }
        }
    };
    load_window();
    if (lane == 0) {
        for (int t = 0; t < NS; ++t) mbar_init(bars + t, 1);
        mbar_init_fence();
    }
    __syncwarp();
    for (int t = 0; t < NS && t < cnt; ++t) post(t, t);
    for (int i = 0; i < cnt; ++i) {
        const int64_t s = s0 + i;
        const int st = i % NS;
        const unsigned char* stage = ring + (size_t)st * L.stage_bytes;
        const unsigned par = (unsigned)((i / NS) & 1);
        if (!mbar_try_wait(bars + st, par)) {  // bounded wait (2 s) for the stage's copies
            const unsigned long long t0 = globaltimer_ns();
            while (!mbar_try_wait(bars + st, par)) {
                if (globaltimer_ns() - t0 > 2000000000ull) {
                    if (lane == 0) atomicExch(&g_stage_timeout, 1);
                    return;
                }
            }
        }
        const int64_t r = s * kSlice + lane;
        const int32_t* hdr = reinterpret_cast<const int32_t*>(stage);
        // every load of the slice first (indices and values from shared memory, x and
        // e4m3 scales from global), then the partial sums in ascending column order
        int w[Q], c[Q][W];
        float v[Q][W], xf[Q][W];
        double vd[F64 ? W : 1], xd[F64 ? W : 1];
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            w[k] = hdr[k];
            const int32_t* cs = reinterpret_cast<const int32_t*>(stage + L.col_off[k]);
#pragma unroll
            for (int l = 0; l < W; ++l) c[k][l] = l < w[k] ? cs[32 * l + lane] : -1;
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const BucketDev& B = M.b[k];
            const unsigned char* vs = stage + L.val_off[k];
            const bool f64 = F64 && k == 0;
            const float sc = (!f64 && B.slicescale) ? __ldg(B.slicescale + s) : B.scale;
#pragma unroll
            for (int l = 0; l < W; ++l) {
                const int cc = c[k][l];
                if (cc >= 0) {
                    if (f64) {
                        vd[F64 ? l : 0] = reinterpret_cast<const double*>(vs)[32 * l + lane];
                        xd[F64 ? l : 0] = (double)__ldg(x + cc);
                    } else {
                        v[k][l] = decode_sm(B, vs, 32 * l + lane, cc, r, sc);
                        xf[k][l] = to_f32<XT>(__ldg(x + cc));
                    }
                }
            }
        }
        constexpr bool F32OUT = std::is_same<YT, float>::value && !F64 && Q <= 2;  // as in k_bspmv_q
        double yi = 0.0;
        float yf = 0.0f;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const BucketDev& B = M.b[k];
            const int32_t* cs = reinterpret_cast<const int32_t*>(stage + L.col_off[k]);
            const unsigned char* vs = stage + L.val_off[k];
            if (F64 && k == 0) {
                double acc = 0.0;
#pragma unroll
                for (int l = 0; l < W; ++l)
                    if (c[k][l] >= 0) acc = __dadd_rn(acc, __dmul_rn(vd[F64 ? l : 0], xd[F64 ? l : 0]));
                for (int l = W; l < w[k]; ++l) {
                    const int cc = cs[32 * l + lane];
                    if (cc >= 0)
                        acc = __dadd_rn(acc, __dmul_rn(reinterpret_cast<const double*>(vs)[32 * l + lane],
                                                       (double)__ldg(x + cc)));
                }
                yi = __dadd_rn(yi, acc);
            } else {
                const float sc = B.slicescale ? __ldg(B.slicescale + s) : B.scale;
                float acc = 0.0f;
#pragma unroll
                for (int l = 0; l < W; ++l)
                    if (c[k][l] >= 0) acc = __fadd_rn(acc, __fmul_rn(v[k][l], xf[k][l]));
                for (int l = W; l < w[k]; ++l) {
                    const int cc = cs[32 * l + lane];
                    if (cc >= 0)
                        acc = __fadd_rn(acc, __fmul_rn(decode_sm(B, vs, 32 * l + lane, cc, r, sc),
                                                       to_f32<XT>(__ldg(x + cc))));
                }
                if constexpr (F32OUT) yf = k == 0 ? acc : __fadd_rn(yf, acc);
            else yi = __dadd_rn(yi, (double)acc);
            }
        }
        __syncwarp();  // every lane is done with this stage
        if (i + NS < cnt) post(i + NS, st);
        if (r < M.n) {
            if constexpr (F32OUT) y[r] = yf;
            else y[r] = from_f64<YT>(yi);
        }
    }
}

// ---------------------------------------------------------------- fixed-format form
// The register form again with the storage format of every bucket fixed at
// compile time (the bucket mixes that occur on the solver's hot path), so that
// decoding needs no run-time dispatch.  Same operations, same order, same bits.
template <int P>
struct FixDec;
template <>
struct FixDec<BSPAI_FP32> {
    static __device__ __forceinline__ float get(const BucketDev& B, int64_t p, float, int, int64_t) {
        return __ldg(reinterpret_cast<const float*>(B.val) + p);
    }
};
template <>
struct FixDec<BSPAI_FP16> {
    static __device__ __forceinline__ float get(const BucketDev& B, int64_t p, float sc, int, int64_t) {
        return __fmul_rn(__half2float(__ldg(reinterpret_cast<const __half*>(B.val) + p)), sc);
    }
};
template <>
struct FixDec<BSPAI_BF16> {
    static __device__ __forceinline__ float get(const BucketDev& B, int64_t p, float, int, int64_t) {
        return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16*>(B.val) + p));
    }
};
template <>
struct FixDec<BSPAI_E4M3> {
    static __device__ __forceinline__ float get(const BucketDev& B, int64_t p, float, int c, int64_t r) {
        __nv_fp8_e4m3 e;
        e.__x = __ldg(reinterpret_cast<const __nv_fp8_storage_t*>(B.val) + p);
        return __fmul_rn(float(e), B.colscale ? __ldg(B.colscale + c) : __ldg(B.rowscale + r));
    }
};

// One row's share of one bucket: slot bounds, then W column indices, then
// values and x entries, then the partial sum (slots beyond W in a plain loop).
template <int P, int W, typename XT>
struct FixRow {
    using V = typename std::conditional<P == BSPAI_FP64, double, float>::type;
    int64_t base;
    int w;
    int c[W];
    V v[W], xv[W];
    __device__ __forceinline__ void ptrs(const BucketDev& B, int64_t s, int lane) {
        const int64_t b0 = __ldg(B.sptr + s);
        base = b0 + lane;
        w = (int)((__ldg(B.sptr + s + 1) - b0) >> 5);
    }
    __device__ __forceinline__ void cols(const BucketDev& B) {
#pragma unroll
        for (int l = 0; l < W; ++l) c[l] = l < w ? __ldg(B.col + base + 32 * l) : -1;
    }
    __device__ __forceinline__ V dec(const BucketDev& B, int64_t p, float sc, int cc, int64_t r) const {
        if constexpr (P == BSPAI_FP64) return __ldg(reinterpret_cast<const double*>(B.val) + p);
        else return FixDec<P>::get(B, p, sc, cc, r);
    }
    __device__ __forceinline__ V xin(const XT* __restrict__ x, int cc) const {
        if constexpr (P == BSPAI_FP64) return (double)__ldg(x + cc);
        else return to_f32<XT>(__ldg(x + cc));
    }
    __device__ __forceinline__ void vals(const BucketDev& B, const XT* __restrict__ x, float sc, int64_t r) {
#pragma unroll
        for (int l = 0; l < W; ++l)
            if (c[l] >= 0) {
                v[l] = dec(B, base + 32 * l, sc, c[l], r);
                xv[l] = xin(x, c[l]);
            }
    }
    // the partial sum y_i^(k): fp64 for an fp64 bucket, fp32 otherwise
    __device__ __forceinline__ V sum(const BucketDev& B, const XT* __restrict__ x, float sc, int64_t r) const {
        if constexpr (P == BSPAI_FP64) {
            double acc = 0.0;
#pragma unroll
            for (int l = 0; l < W; ++l)
                if (c[l] >= 0) acc = __dadd_rn(acc, __dmul_rn(v[l], xv[l]));
            for (int l = W; l < w; ++l) {
                const int cc = __ldg(B.col + base + 32 * l);
                if (cc >= 0) acc = __dadd_rn(acc, __dmul_rn(dec(B, base + 32 * l, sc, cc, r), xin(x, cc)));
            }
            return acc;
        } else {
            float acc = 0.0f;
#pragma unroll
            for (int l = 0; l < W; ++l)
                if (c[l] >= 0) acc = __fadd_rn(acc, __fmul_rn(v[l], xv[l]));
            for (int l = W; l < w; ++l) {
                const int cc = __ldg(B.col + base + 32 * l);
                if (cc >= 0) acc = __fadd_rn(acc, __fmul_rn(dec(B, base + 32 * l, sc, cc, r), xin(x, cc)));
            }
            return acc;
        }
    }
};

// P1 < 0: one bucket.  The register cap (min blocks per SM) buys occupancy:
// with a handful of loads in flight per thread, more resident warps is what
// keeps more bytes in flight.
template <int P0, int W0, int P1>
struct FixMinBlocks {
    static constexpr int value = P1 < 0 ? (W0 > 4 ? 4 : (P0 == BSPAI_FP64 ? 6 : 8)) : (W0 > 4 ? 4 : 6);
};

template <typename XT, typename YT, int P0, int W0, int P1, int W1>
__global__ void __launch_bounds__(256, FixMinBlocks<P0, W0, P1>::value) k_bspmv_fix(const __grid_constant__ BMDev M, const XT* __restrict__ x,
                                                   YT* __restrict__ y, const int* __restrict__ jd, int64_t ldx,
                                                   int64_t ldy, int yoff) {
    if (jd) {
        if (jd[1]) return;
        const int64_t j = jd[0];
        x += j * ldx;
        y += (j + yoff) * ldy;
    }
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (int64_t)ceil_div(M.n, kSlice) * kSlice) return;
    const int64_t s = r >> 5;
    const int lane = (int)(r & 31);
    FixRow<P0, W0, XT> a;
    FixRow<(P1 < 0 ? BSPAI_FP32 : P1), W1, XT> b;
    const float sc0 = M.b[0].slicescale ? __ldg(M.b[0].slicescale + s) : M.b[0].scale;
    float sc1 = 1.0f;
    a.ptrs(M.b[0], s, lane);
    if constexpr (P1 >= 0) {
        sc1 = M.b[1].slicescale ? __ldg(M.b[1].slicescale + s) : M.b[1].scale;
        b.ptrs(M.b[1], s, lane);
    }
    a.cols(M.b[0]);
    if constexpr (P1 >= 0) b.cols(M.b[1]);
    a.vals(M.b[0], x, sc0, r);
    if constexpr (P1 >= 0) b.vals(M.b[1], x, sc1, r);
    constexpr bool narrow = P0 != BSPAI_FP64 && P1 != BSPAI_FP64;
    if constexpr (narrow && std::is_same<YT, float>::value) {
        // fp32 partials, fp32 result: fl32(fl64(0 + a)) = a, and for two
        // partials fl32(fl64(a + b)) = fl32(a + b) (double rounding through
        // 53 >= 2 * 24 + 2 bits is innocuous), so the fp64 sum of Alg 2.3 in
        // bucket order gives these bits without fp64 arithmetic
        float yf = a.sum(M.b[0], x, sc0, r);
        if constexpr (P1 >= 0) yf = __fadd_rn(yf, b.sum(M.b[1], x, sc1, r));
        if (r < M.n) y[r] = yf;
    } else {
        double yi = __dadd_rn(0.0, (double)a.sum(M.b[0], x, sc0, r));
        if constexpr (P1 >= 0) yi = __dadd_rn(yi, (double)b.sum(M.b[1], x, sc1, r));
        if (r < M.n) y[r] = from_f64<YT>(yi);
    }
}

template <typename XT, typename YT>
using FixFn = void (*)(BMDev, const XT*, YT*, const int*, int64_t, int64_t, int);

// the compiled bucket mixes: one bucket (fp32, fp64, fp16), or two
// consecutive stored formats (fp16 + e4m3, fp32 + fp16, fp64 + fp32)
template <typename XT, typename YT>
static FixFn<XT, YT> pick_fix(const BMDev& M, int W) {
#define BSPAI_FIX1(p, w) \
    if (M.q == 1 && M.b[0].prec == p && W == w) return k_bspmv_fix<XT, YT, p, w, -1, 4>;
#define BSPAI_FIX2(p0, p1, w) \
    if (M.q == 2 && M.b[0].prec == p0 && M.b[1].prec == p1 && W == w) return k_bspmv_fix<XT, YT, p0, w, p1, w>;
    BSPAI_FIX1(BSPAI_FP32, 4) BSPAI_FIX1(BSPAI_FP32, 8) BSPAI_FIX1(BSPAI_FP64, 4) BSPAI_FIX1(BSPAI_FP64, 8)
    BSPAI_FIX1(BSPAI_FP16, 4) BSPAI_FIX1(BSPAI_FP16, 8)
    BSPAI_FIX2(BSPAI_FP16, BSPAI_E4M3, 4) BSPAI_FIX2(BSPAI_FP16, BSPAI_E4M3, 8)
    BSPAI_FIX2(BSPAI_FP32, BSPAI_FP16, 4) BSPAI_FIX2(BSPAI_FP32, BSPAI_FP16, 8)
    BSPAI_FIX2(BSPAI_FP64, BSPAI_FP32, 4) BSPAI_FIX2(BSPAI_FP64, BSPAI_FP32, 8)
#undef BSPAI_FIX1
#undef BSPAI_FIX2
    return nullptr;
}

// ---------------------------------------------------------------- packed form
// The product on buckets in the packed slot arrangement (a row's slots in
// groups of four consecutive elements).  Per group and lane, one vector load
// brings the four column indices (16 B of int32 or 8 B of 16-bit differences)
// and one the four stored values (32 / 16 / 8 / 8 / 4 B in fp64 / fp32 / fp16 /
// bf16 / e4m3), both streamed past L1 (ld.global.cs) so that L1 keeps the
// gathered x entries and e4m3 column scales; a warp's loads are 128
// consecutive elements.  Then x (and the column scales) are gathered and each
// bucket's partial sum is formed in ascending column order with the same
// operations as the other forms: the same bits.

template <int P>
struct PkRaw;  // the four stored values of one group, converted exactly to V
template <>
struct PkRaw<BSPAI_FP64> {
    static __device__ __forceinline__ void get(const void* val, int64_t g, double v[4]) {
        const double2 a = __ldcs(reinterpret_cast<const double2*>(reinterpret_cast<const double*>(val) + g));
        const double2 b = __ldcs(reinterpret_cast<const double2*>(reinterpret_cast<const double*>(val) + g + 2));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};
template <>
struct PkRaw<BSPAI_FP32> {
    static __device__ __forceinline__ void get(const void* val, int64_t g, float v[4]) {
        const float4 a = __ldcs(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(val) + g));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
};
template <>
struct PkRaw<BSPAI_FP16> {
    static __device__ __forceinline__ void get(const void* val, int64_t g, float v[4]) {
        const uint2 u = __ldcs(reinterpret_cast<const uint2*>(reinterpret_cast<const __half*>(val) + g));
        const __half2 h01 = *reinterpret_cast<const __half2*>(&u.x), h23 = *reinterpret_cast<const __half2*>(&u.y);
        v[0] = __low2float(h01); v[1] = __high2float(h01); v[2] = __low2float(h23); v[3] = __high2float(h23);
    }
};
template <>
struct PkRaw<BSPAI_BF16> {
    static __device__ __forceinline__ void get(const void* val, int64_t g, float v[4]) {
        const uint2 u = __ldcs(reinterpret_cast<const uint2*>(reinterpret_cast<const __nv_bfloat16*>(val) + g));
        v[0] = __uint_as_float(u.x << 16); v[1] = __uint_as_float(u.x & 0xffff0000u);
        v[2] = __uint_as_float(u.y << 16); v[3] = __uint_as_float(u.y & 0xffff0000u);
    }
};
template <>
struct PkRaw<BSPAI_E4M3> {
    static __device__ __forceinline__ void get(const void* val, int64_t g, float v[4]) {
        const unsigned u = __ldcs(reinterpret_cast<const unsigned*>(reinterpret_cast<const __nv_fp8_storage_t*>(val) + g));
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            __nv_fp8_e4m3 f;
            f.__x = (__nv_fp8_storage_t)((u >> (8 * e)) & 0xffu);
            v[e] = float(f);
        }
    }
};

// one row's share of one packed bucket
template <int P, typename XT, bool I16>
struct PkRow {
    using V = typename std::conditional<P == BSPAI_FP64, double, float>::type;
    int64_t sb;  // first element of the row's slice
    int ng;      // groups of four slots per row in the slice
    int c[4];
    V v[4], xv[4];
    // (a uniform slice width needs no load: the matrix stream starts at once)
    __device__ __forceinline__ void ptrs(const BucketDev& B, int64_t s) {
        if (B.ellw > 0) {
            sb = s * ((int64_t)B.ellw << 5);
            ng = B.ellw >> 2;
        } else {
            sb = __ldg(B.sptr + s);
            ng = (int)((__ldg(B.sptr + s + 1) - sb) >> 7);
        }
    }
    // indices and stored values of group grp (none when the slice has no
    // group); an fp16 value times its bucket's scale (exact: a power of two)
    __device__ __forceinline__ void load(const BucketDev& B, int grp, int lane, int64_t r, float sc) {
        if (grp >= ng) {
            c[0] = c[1] = c[2] = c[3] = -1;
            return;
        }
        const int64_t g = sb + ((int64_t)grp << 7) + (lane << 2);
        if constexpr (I16) {
            const uint2 u = __ldcs(reinterpret_cast<const uint2*>(B.col16 + g));
            const int d0 = (int16_t)(u.x & 0xffffu), d1 = (int16_t)(u.x >> 16), d2 = (int16_t)(u.y & 0xffffu),
                      d3 = (int16_t)(u.y >> 16);
            c[0] = d0 == kCol16Pad ? -1 : (int)r + d0;
            c[1] = d1 == kCol16Pad ? -1 : (int)r + d1;
            c[2] = d2 == kCol16Pad ? -1 : (int)r + d2;
            c[3] = d3 == kCol16Pad ? -1 : (int)r + d3;
        } else {
            const int4 u = __ldcs(reinterpret_cast<const int4*>(B.col + g));
            c[0] = u.x; c[1] = u.y; c[2] = u.z; c[3] = u.w;
        }
        PkRaw<P>::get(B.val, g, v);
        if constexpr (P == BSPAI_FP16) {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = __fmul_rn(v[e], sc);
        }
    }
    // x entries; an e4m3 value times its scale (per column of M, or per row of
    // a transposed M; exact: a power of two)
    __device__ __forceinline__ void gather(const BucketDev& B, const XT* __restrict__ x, int64_t r) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (c[e] >= 0) {
                if constexpr (P == BSPAI_FP64) xv[e] = (double)__ldg(x + c[e]);
                else xv[e] = to_f32<XT>(__ldg(x + c[e]));
                if constexpr (P == BSPAI_E4M3)
                    v[e] = __fmul_rn(v[e], B.colscale ? __ldg(B.colscale + c[e]) : __ldg(B.rowscale + r));
            }
    }
    // add the group's products to acc in slot order
    __device__ __forceinline__ void accumulate(V& acc) const {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (c[e] >= 0) {
                if constexpr (P == BSPAI_FP64) acc = __dadd_rn(acc, __dmul_rn(v[e], xv[e]));
                else acc = __fadd_rn(acc, __fmul_rn(v[e], xv[e]));
            }
    }
    // the partial sum y_i^(k): group 0 (already loaded and gathered), then the
    // rest (ONE: the slice has at most one group)
    template <bool ONE>
    __device__ __forceinline__ V sum(const BucketDev& B, const XT* __restrict__ x, float sc, int lane, int64_t r) {
        V acc = V(0);
        accumulate(acc);
        if constexpr (!ONE) {
            for (int grp = 1; grp < ng; ++grp) {
                load(B, grp, lane, r, sc);
                gather(B, x, r);
                accumulate(acc);
            }
        }
        return acc;
    }
};

template <int P0, int P1, bool ONE>
struct PkMinBlocks {
    static constexpr int value = (P0 == BSPAI_FP64 || P1 == BSPAI_FP64) ? 4 : (ONE ? 8 : 4);
};

// P1 < 0: one bucket.  ONE: every row of the matrix has at most four slots
// per bucket (one group), so the kernel has no loop and few registers: eight
// 256-thread blocks fit per SM (four with the loop or with an fp64 bucket).
template <typename XT, typename YT, int P0, int P1, bool I16, bool ONE>
__global__ void __launch_bounds__(256, PkMinBlocks<P0, P1, ONE>::value)
    k_bspmv_pk(const __grid_constant__ BMDev M, const XT* __restrict__ x, YT* __restrict__ y,
               const int* __restrict__ jd, int64_t ldx, int64_t ldy, int yoff) {
    if (jd) {
        if (jd[1]) return;
        const int64_t j = jd[0];
        x += j * ldx;
        y += (j + yoff) * ldy;
    }
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (int64_t)ceil_div(M.n, kSlice) * kSlice) return;
    const int64_t s = r >> 5;
    const int lane = (int)(r & 31);
    PkRow<P0, XT, I16> a;
    PkRow<(P1 < 0 ? BSPAI_FP32 : P1), XT, I16> b;
    const float sc0 = M.b[0].slicescale ? __ldg(M.b[0].slicescale + s) : M.b[0].scale;
    float sc1 = 1.0f;
    a.ptrs(M.b[0], s);
    if constexpr (P1 >= 0) {
        sc1 = M.b[1].slicescale ? __ldg(M.b[1].slicescale + s) : M.b[1].scale;
        b.ptrs(M.b[1], s);
    }
    a.load(M.b[0], 0, lane, r, sc0);
    if constexpr (P1 >= 0) b.load(M.b[1], 0, lane, r, sc1);
    a.gather(M.b[0], x, r);
    if constexpr (P1 >= 0) b.gather(M.b[1], x, r);
    constexpr bool narrow = P0 != BSPAI_FP64 && P1 != BSPAI_FP64;
    if constexpr (narrow && std::is_same<YT, float>::value) {
        // as in k_bspmv_fix: the fp32 result of at most two fp32 partials needs no fp64 arithmetic
        float yf = a.template sum<ONE>(M.b[0], x, sc0, lane, r);
        if constexpr (P1 >= 0) yf = __fadd_rn(yf, b.template sum<ONE>(M.b[1], x, sc1, lane, r));
        if (r < M.n) y[r] = yf;
    } else {
        double yi = __dadd_rn(0.0, (double)a.template sum<ONE>(M.b[0], x, sc0, lane, r));
        if constexpr (P1 >= 0) yi = __dadd_rn(yi, (double)b.template sum<ONE>(M.b[1], x, sc1, lane, r));
        if (r < M.n) y[r] = from_f64<YT>(yi);
    }
}

// One packed bucket whose rows have at most eight slots (two groups, e.g. a
// 7-point stencil): both groups' indices and values are loaded before any
// gather, then the partial sum is formed group by group in slot order.
template <typename XT, typename YT, int P, bool I16>
__global__ void __launch_bounds__(256, P == BSPAI_FP64 ? 4 : 6)
    k_bspmv_pk2g(const __grid_constant__ BMDev M, const XT* __restrict__ x, YT* __restrict__ y,
                 const int* __restrict__ jd, int64_t ldx, int64_t ldy, int yoff) {
    if (jd) {
        if (jd[1]) return;
        const int64_t j = jd[0];
        x += j * ldx;
        y += (j + yoff) * ldy;
    }
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (int64_t)ceil_div(M.n, kSlice) * kSlice) return;
    const int64_t s = r >> 5;
    const int lane = (int)(r & 31);
    const float sc = M.b[0].slicescale ? __ldg(M.b[0].slicescale + s) : M.b[0].scale;
    PkRow<P, XT, I16> g0, g1;
    g0.ptrs(M.b[0], s);
    g1.sb = g0.sb;
    g1.ng = g0.ng;
    g0.load(M.b[0], 0, lane, r, sc);
    g1.load(M.b[0], 1, lane, r, sc);
    g0.gather(M.b[0], x, r);
    g1.gather(M.b[0], x, r);
    typename PkRow<P, XT, I16>::V acc = 0;
    g0.accumulate(acc);
    g1.accumulate(acc);
    if constexpr (P != BSPAI_FP64 && std::is_same<YT, float>::value) {
        if (r < M.n) y[r] = acc;  // fl32(fl64(0 + a)) = a
    } else {
        if (r < M.n) y[r] = from_f64<YT>(__dadd_rn(0.0, (double)acc));
    }
}

// the compiled packed mixes (as pick_fix), for either index width; null if
// the buckets are not all packed alike or the mix is not compiled
template <typename XT, typename YT, bool I16, bool ONE>
static FixFn<XT, YT> pick_pk_mix(const BMDev& M) {
#define BSPAI_PK1(p) \
    if (M.q == 1 && M.b[0].prec == p) return k_bspmv_pk<XT, YT, p, -1, I16, ONE>;
#define BSPAI_PK2(p0, p1) \
    if (M.q == 2 && M.b[0].prec == p0 && M.b[1].prec == p1) return k_bspmv_pk<XT, YT, p0, p1, I16, ONE>;
    BSPAI_PK1(BSPAI_FP32) BSPAI_PK1(BSPAI_FP64) BSPAI_PK1(BSPAI_FP16) BSPAI_PK1(BSPAI_BF16) BSPAI_PK1(BSPAI_E4M3)
    BSPAI_PK2(BSPAI_FP16, BSPAI_E4M3) BSPAI_PK2(BSPAI_FP32, BSPAI_FP16) BSPAI_PK2(BSPAI_FP64, BSPAI_FP32)
    BSPAI_PK2(BSPAI_FP32, BSPAI_E4M3) BSPAI_PK2(BSPAI_FP16, BSPAI_BF16)
#undef BSPAI_PK1
#undef BSPAI_PK2
    return nullptr;
}

template <typename XT, typename YT>
static FixFn<XT, YT> pick_pk(const BMDev& M) {
    int maxw = 0;
    for (int k = 0; k < M.q; ++k) {
        if (!M.b[k].packed || (M.b[k].col16 != nullptr) != (M.b[0].col16 != nullptr) || M.b[k].maxw < 0)
            return nullptr;
        maxw = M.b[k].maxw > maxw ? M.b[k].maxw : maxw;
    }
    const bool i16 = M.b[0].col16 != nullptr, one = maxw <= 4;
    if (M.q == 1 && !one && maxw <= 8) {
        const int p = M.b[0].prec;
        if (p == BSPAI_FP32) return i16 ? k_bspmv_pk2g<XT, YT, BSPAI_FP32, true> : k_bspmv_pk2g<XT, YT, BSPAI_FP32, false>;
        if (p == BSPAI_FP64) return i16 ? k_bspmv_pk2g<XT, YT, BSPAI_FP64, true> : k_bspmv_pk2g<XT, YT, BSPAI_FP64, false>;
        if (p == BSPAI_FP16) return i16 ? k_bspmv_pk2g<XT, YT, BSPAI_FP16, true> : k_bspmv_pk2g<XT, YT, BSPAI_FP16, false>;
    }
    if (i16) return one ? pick_pk_mix<XT, YT, true, true>(M) : pick_pk_mix<XT, YT, true, false>(M);
    return one ? pick_pk_mix<XT, YT, false, true>(M) : pick_pk_mix<XT, YT, false, false>(M);
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
    d.b[0].maxw = S.maxw;
    d.b[0].packed = S.packed;
    d.b[0].col16 = S.col16;
    d.b[0].ellw = S.ellw;
    return d;
}


BMDev up_view(const bspai_matrix* A, int up) {
    if (up == BSPAI_FP32 && A->pval32) return single_bucket_view(A->psell, A->pval32, BSPAI_FP32);
    return single_bucket_view(A->sell, up == BSPAI_FP64 ? (const void*)A->val64 : (const void*)A->val32, up);
}

template <typename XT, typename YT>
using TmaFn = void (*)(BMDev, const XT*, YT*, const int*, int64_t, int64_t, int, StageLayout);

template <typename XT, typename YT>
static TmaFn<XT, YT> pick_tma(int Q, int W, bool f64) {
#define BSPAI_PICK_TMA(q, w)                                                                  \
    if (Q == q && W == w) return f64 ? (TmaFn<XT, YT>)k_bspmv_tma<XT, YT, q, w, true>          \
                                     : (TmaFn<XT, YT>)k_bspmv_tma<XT, YT, q, w, false>;
    BSPAI_PICK_TMA(1, 4) BSPAI_PICK_TMA(1, 8) BSPAI_PICK_TMA(2, 4) BSPAI_PICK_TMA(2, 8) BSPAI_PICK_TMA(3, 4)
    BSPAI_PICK_TMA(4, 4)
#undef BSPAI_PICK_TMA
    return nullptr;
}

static int prec_value_bytes(int prec) {
    switch (prec) {
    case BSPAI_FP64: return 8;
    case BSPAI_FP32: return 4;
    case BSPAI_FP16:
    case BSPAI_BF16: return 2;
    case BSPAI_E4M3: return 1;
    default: return 0;
    }
}

constexpr int kTmaWarps = 8;
static std::atomic<int> g_spmv_form{BSPAI_SPMV_AUTO};
static int align16i(int v) { return (v + 15) & ~15; }

// Stage layout for the compacted buckets of M, or false when the TMA form does
// not apply (unknown slice widths, misaligned arrays, too few slices to keep
// every warp busy, or a stage ring that does not fit).
static bool tma_plan(const BMDev& M, StageLayout* L, size_t* smem) {
    if (M.q < 1 || M.q > 4) return false;
    for (int k = 0; k < M.q; ++k)  // the staged form reads the plain arrangement with int32 columns
        if (M.b[k].packed || M.b[k].col16) return false;
    if (ceil_div(M.n, kSlice) < (int64_t)2 * kTmaWarps * num_sms()) return false;
    int off = kStageHeader;
    for (int k = 0; k < M.q; ++k) {
        const BucketDev& B = M.b[k];
        const int vb = prec_value_bytes(B.prec);
        if (B.maxw < 0 || vb == 0) return false;
        if (((uintptr_t)B.col & 15) || ((uintptr_t)B.val & 15)) return false;
        L->vbytes[k] = vb;
        L->col_off[k] = off;
        off += align16i(128 * B.maxw);
        L->val_off[k] = off;
        off += align16i(32 * B.maxw * vb);
    }
    L->stage_bytes = align16i(off);
    // four stages per warp where four 8-warp blocks still fit on an SM, else fewer
    for (int ns : {4, 3, 2}) {
        const size_t need = (size_t)kTmaWarps * ns * (8 + (size_t)L->stage_bytes);
        if (need <= 56 * 1024 || (ns == 2 && need <= 112 * 1024)) {
            L->ns = ns;
            *smem = need;
            return true;
        }
    }
    return false;
}

template <typename XT, typename YT>
static bool launch_tma(const BMDev& M, const XT* x, YT* y, const int* jd, int64_t ldx, int64_t ldy, int yoff,
                       cudaStream_t s) {
    StageLayout L{};
    size_t smem = 0;
    if (!tma_plan(M, &L, &smem)) return false;
    int maxw = 0;
    for (int k = 0; k < M.q; ++k) maxw = M.b[k].maxw > maxw ? M.b[k].maxw : maxw;
    TmaFn<XT, YT> fn = pick_tma<XT, YT>(M.q, (maxw > 4 && M.q <= 2) ? 8 : 4, M.b[0].prec == BSPAI_FP64);
    if (!fn) return false;
    // per-instance opt-in to the dynamic shared memory, and its occupancy
    static std::mutex mu;
    static std::map<std::pair<const void*, size_t>, int> occ_cache;
    int occ = 0;
    {
        std::lock_guard<std::mutex> g(mu);
        auto key = std::make_pair((const void*)fn, smem);
        auto it = occ_cache.find(key);
        if (it == occ_cache.end()) {
            if (cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32 * kTmaWarps, smem))
                occ = 0;
            occ_cache[key] = occ;
        } else {
            occ = it->second;
        }
    }
    if (occ < 1) return false;
    const unsigned grid = (unsigned)(num_sms() * occ);
    fn<<<grid, 32 * kTmaWarps, smem, s>>>(M, x, y, jd, ldx, ldy, yoff, L);
    return true;
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
    const int form = g_spmv_form.load(std::memory_order_relaxed);
    if (form == BSPAI_SPMV_AUTO && M.q >= 1 && M.b[0].packed) {
        if (FixFn<XT, YT> pf = pick_pk<XT, YT>(M)) {
            pf<<<grid, 256, 0, s>>>(M, x, y, jd, ldx, ldy, yoff);
            return;
        }
    }
    if (form == BSPAI_SPMV_AUTO && known && !M.b[0].packed) {
        if (FixFn<XT, YT> ff = pick_fix<XT, YT>(M, W)) {
            ff<<<grid, 256, 0, s>>>(M, x, y, jd, ldx, ldy, yoff);
            return;
        }
    }
    if (form == BSPAI_SPMV_STAGED && launch_tma<XT, YT>(M, x, y, jd, ldx, ldy, yoff, s)) return;
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
        d.b[k].packed = b[k].packed;
        d.b[k].col16 = b[k].col16;
        d.b[k].ellw = b[k].ellw;
    }
    return d;
}

namespace bspai {
// BSPAI_TIMEOUT if a TMA-staged SpMV gave up waiting since the last call (and
// clears the flag); synchronises stream s
int stage_timeout_take(cudaStream_t s) {
    int h = 0, z = 0;
    CUDA_TRY(cudaMemcpyFromSymbolAsync(&h, g_stage_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (!h) return BSPAI_OK;
    CUDA_TRY(cudaMemcpyToSymbolAsync(g_stage_timeout, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return set_error(BSPAI_TIMEOUT, "spmv: a shared-memory stage was not filled within its time limit");
}
// y = M x with M in u_f = fp16 (Alg 3.1's x0 = M b in the (half, single,
// double) setting): x_j rounded once from fp64 to fp16, every product and
// partial sum an fp16 operation (the fp32 operation rounded once more, exact
// for the product of two fp16 values and correctly rounded for the sum by the
// double-rounding theorem, 24 >= 2 * 11 + 2), in ascending column order; y
// stored in fp64.  One thread per row of the SELL-32 layout: the 32 rows of a
// slice read consecutive slots.
__global__ void k_spmv_uf16(int n, const int64_t* __restrict__ sptr, const int32_t* __restrict__ col,
                            const float* __restrict__ val, const int32_t* __restrict__ rowlen,
                            const double* __restrict__ x, double* __restrict__ y) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t b = sptr[r >> 5] + (r & 31);
    const int len = rowlen[r];
    float acc = 0.0f;
    for (int l = 0; l < len; ++l) {
        const int64_t p = b + (int64_t)l * kSlice;
        const float xv = __half2float(__double2half(x[col[p]]));
        const float pr = __half2float(__float2half_rn(__fmul_rn(val[p], xv)));
        acc = __half2float(__float2half_rn(__fadd_rn(acc, pr)));
    }
    y[r] = (double)acc;
}

int launch_apply_uf(const bspai_spai* M, const double* x, double* y, cudaStream_t s) {
    if (M->uf == BSPAI_FP16) {
        if (M->n <= 0) return BSPAI_OK;
        k_spmv_uf16<<<(unsigned)ceil_div(M->n, 256), 256, 0, s>>>(M->n, M->sell.sptr, M->sell.col, M->val,
                                                                  M->rowlen, x, y);
        note_launch();
        CUDA_LAUNCH_CHECK();
        return BSPAI_OK;
    }
    return launch_bspmv(single_bucket_view(M->sell, M->val, BSPAI_FP32), x, BSPAI_FP64, y, BSPAI_FP64, s);
}
}  // namespace bspai

extern "C" {

int bspai_set_spmv_form(int form) {
    if (form != BSPAI_SPMV_AUTO && form != BSPAI_SPMV_REGISTERS && form != BSPAI_SPMV_STAGED)
        return set_error(BSPAI_ERR_INVALID, "bspai_set_spmv_form: unknown form %d", form);
    g_spmv_form.store(form);
    return BSPAI_OK;
}

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
    return launch_apply_uf(M, x, y, (cudaStream_t)s);
}

int bspai_spmv_up(bspai_A_h A, const float* v, float* w, bspai_stream_t s) {
    if (!A || A->magic != kMagicA) return set_error(BSPAI_ERR_INVALID, "bspai_spmv_up: bad handle");
    if (!v || !w) return set_error(BSPAI_ERR_INVALID, "bspai_spmv_up: null vector");
    ProfScope ps(BSPAI_K_SPMV_A, (cudaStream_t)s);
    return launch_bspmv(up_view(A, BSPAI_FP32), v, BSPAI_FP32, w, BSPAI_FP32, (cudaStream_t)s);
}

}  // extern "C"
