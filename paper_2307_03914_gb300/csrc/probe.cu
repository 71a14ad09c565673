// probe.cu -- measured issue rate of the SM's plain (non-tensor) fused
// multiply-add pipes in fp32 and fp64.  These are the denominators of the ALU
// rooflines of the kernels that arithmetic, not memory, bounds: the SPAI build
// (Householder least squares in u_f = fp32) and the Dot2 residual (fp64).  The
// paper has no counterpart; it is a measurement aid.
//
// Every thread runs eight independent chains of dependent FMAs (enough to
// cover the pipe latency at full occupancy), on a grid of eight 256-thread
// blocks per SM.  The chains' results are folded into one store that depends
// on all of them, so nothing is removed by the compiler.
#include "common.cuh"

namespace bspai {

template <typename T>
__device__ __forceinline__ T fma_rn(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_rn<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double fma_rn<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T* __restrict__ out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < 8; ++c) x[c] = fma_rn<T>(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    // a and b keep the chains bounded (|a| < 1); the store is taken only for an
    // impossible value, but the compiler cannot know that
    if (s == (T)-12345.678) out[blockIdx.x] = s;
}

template <typename T>
static int probe(int iters, cudaStream_t s, double* fma_per_s, float* ms_out) {
    const int grid = 8 * num_sms();
    T* out = nullptr;
    BSPAI_TRY(dalloc_t(&out, (size_t)grid, s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = BSPAI_OK;
    cudaError_t e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    if (!e) {
        k_fma_probe<T><<<grid, 256, 0, s>>>(out, iters / 8 > 0 ? iters / 8 : 1, (T)0.999, (T)1e-4);  // warm-up
        note_launch();
        e = cudaEventRecord(e0, s);
    }
    if (!e) {
        k_fma_probe<T><<<grid, 256, 0, s>>>(out, iters, (T)0.999, (T)1e-4);
        note_launch();
        e = cudaGetLastError();
    }
    if (!e) e = cudaEventRecord(e1, s);
    if (!e) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e) rc = cuda_error(e, "fma probe", __FILE__, __LINE__);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dfree(out, s);
    if (rc) return rc;
    // 32 FMAs per thread per iteration
    *fma_per_s = (double)grid * 256.0 * 32.0 * (double)iters / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return BSPAI_OK;
}

}  // namespace bspai

using namespace bspai;

extern "C" {

int bspai_probe_fma(bspai_prec_t prec, int32_t iters, bspai_stream_t st, double* fma_per_s, float* ms) {
    if (!fma_per_s) return set_error(BSPAI_ERR_INVALID, "bspai_probe_fma: null output");
    if (iters < 8 || iters > (1 << 24)) return set_error(BSPAI_ERR_INVALID, "bspai_probe_fma: iters = %d", iters);
    cudaStream_t s = (cudaStream_t)st;
    if (prec == BSPAI_FP32) return probe<float>(iters, s, fma_per_s, ms);
    if (prec == BSPAI_FP64) return probe<double>(iters, s, fma_per_s, ms);
    return set_error(BSPAI_ERR_UNSUPPORTED, "bspai_probe_fma: prec must be FP32 or FP64");
}

}  // extern "C"
