// common.cuh -- internal declarations shared by the libbspai.so translation units.
//
// Storage layout used by every sparse kernel: SELL-32 ("sliced ELLPACK" with
// slices of 32 consecutive rows).  Slice s covers rows 32s..32s+31; its entries
// occupy slots [sptr[s], sptr[s+1]) with sptr[s+1]-sptr[s] = 32 * width_s, and
// entry l of row r sits at slot sptr[r/32] + 32*l + r%32.  One warp handles one
// slice, one thread one row: the 32 lanes read 32 consecutive slots per step
// (fully coalesced), and each row is still accumulated sequentially in
// ascending column order.  Padding slots carry column -1 and value 0.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "bspai.h"

namespace bspai {

constexpr int kSlice = 32;

// ------------------------------------------------------------------ errors
int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what, const char* file, int line);

#define CUDA_TRY(expr)                                                          \
    do {                                                                        \
        cudaError_t _e = (expr);                                                \
        if (_e != cudaSuccess) return ::bspai::cuda_error(_e, #expr, __FILE__, __LINE__); \
    } while (0)

#define CUDA_LAUNCH_CHECK() CUDA_TRY(cudaGetLastError())

#define BSPAI_TRY(expr)                                                         \
    do {                                                                        \
        int _s = (expr);                                                        \
        if (_s != BSPAI_OK) return _s;                                          \
    } while (0)

// ------------------------------------------------------------------ memory
// Stream-ordered device allocation from the device's default memory pool
// (pooled: repeated solves do not return memory to the driver).
int dalloc(void** p, size_t bytes, cudaStream_t s);
template <typename T>
inline int dalloc_t(T** p, size_t count, cudaStream_t s) {
    return dalloc(reinterpret_cast<void**>(p), count * sizeof(T), s);
}
void dfree(void* p, cudaStream_t s);

// ------------------------------------------------------------------ handles
enum : uint32_t {
    kMagicA = 0xB5A10001u,
    kMagicM = 0xB5A10002u,
    kMagicBM = 0xB5A10003u,
    kMagicDead = 0xDEADBEEFu
};

// Sliced ELL with 32-row slices.  Slice s holds its rows' slots in
// [sptr[s], sptr[s + 1]), (sptr[s + 1] - sptr[s]) / 32 slots per row, each
// row's entries first in ascending column order, then padding.  Two
// arrangements inside a slice (sell_slot):
//   plain:  slot l of lane t at sptr[s] + 32 l + t (a warp's loads of slot l
//           are 32 consecutive elements);
//   packed: the slots of a row in groups of four consecutive elements,
//           slot l of lane t at sptr[s] + 128 (l / 4) + 4 t + l % 4, slice
//           widths a multiple of four (one 4-element vector load per lane and
//           group; a warp's load is 128 consecutive elements).
// Column indices are int32 (col; -1 = padding) or, when every entry of the
// structure satisfies |c - r| <= 32767, 16-bit differences c - r to the row r
// (col16; INT16_MIN = padding, col = null).
struct Sell {
    int32_t n = 0;
    int32_t nslices = 0;
    int64_t slots = 0;
    int64_t* sptr = nullptr;   // nslices + 1
    int32_t* col = nullptr;    // slots, -1 = padding (null when col16 is used)
    int32_t maxw = -1;         // widest slice in slots per row (-1: unknown)
    int32_t packed = 0;        // 1: packed arrangement (groups of four slots per row)
    int16_t* col16 = nullptr;  // slots of 16-bit column differences c - r, or null
    int32_t ellw = 0;          // > 0: every slice has this width (sptr[s] = 32 ellw s)
};

constexpr int16_t kCol16Pad = -32768;

// element index of slot l of the row in lane `lane` of a slice starting at sbase
__host__ __device__ __forceinline__ int64_t sell_slot(int64_t sbase, int lane, int l, int packed) {
    return packed ? sbase + ((int64_t)(l >> 2) << 7) + (lane << 2) + (l & 3) : sbase + ((int64_t)l << 5) + lane;
}
// column of slot p of row r (-1: padding)
__device__ __forceinline__ int sell_col(const int32_t* col, const int16_t* col16, int64_t p, int64_t r) {
    if (col16) {
        const int d = col16[p];
        return d == kCol16Pad ? -1 : (int)(r + d);
    }
    return col[p];
}

// Device view of one precision bucket for the SpMV kernels.
struct BucketDev {
    int32_t prec;              // bspai_prec_t
    float scale;               // fp16 bucket: power-of-two scale (else 1)
    const int64_t* sptr;
    const int32_t* col;
    const void* val;           // typed by prec
    const float* colscale;     // e4m3 bucket: per-column scale (else null)
    const float* rowscale;     // e4m3 bucket of a transposed M: per-row scale (else null)
    const float* slicescale;   // fp16 bucket of a batch: per-slice scale (else null: use scale)
    int64_t nnz;               // entries in the bucket (-1: unknown)
    int32_t maxw;              // widest slice of the bucket in slots per row (-1: unknown)
    int32_t packed;            // slot arrangement (Sell::packed)
    const int16_t* col16;      // 16-bit column differences (Sell::col16), or null: col
    int32_t ellw;              // uniform slice width (Sell::ellw), or 0
};

struct BMDev {
    int32_t n;
    int32_t q;
    BucketDev b[8];
};

}  // namespace bspai

struct bspai_matrix {
    uint32_t magic;
    cudaStream_t stream;
    int32_t n;
    int64_t nnz;
    bspai::Sell sell;
    double* val64 = nullptr;   // A in fp64 (residual, u_r)
    float* val32 = nullptr;    // A rounded to fp32 (u_p)
    double* norm_inf = nullptr;// device scalar ||A||_inf
    int32_t* rowlen = nullptr; // entries per row (null for a transposed A)
    int32_t* csr_row_ptr = nullptr; // copy of A's CSR row pointers (null for a transposed A)
    bspai::Sell psell;         // A's structure in the packed slot arrangement (A v in u_p = fp32)
    float* pval32 = nullptr;   // A rounded to fp32 in psell's slots
};

struct bspai_spai {
    uint32_t magic;
    cudaStream_t stream;
    int32_t n;
    int64_t nnz;
    bspai::Sell sell;          // structure of the pattern (rows of M)
    int32_t* rowlen = nullptr; // entries per row
    int32_t* csr_row_ptr = nullptr;
    float* val = nullptr;      // M's values in u_f (fp32, or fp16 values held in fp32)
    int32_t uf = BSPAI_FP32;   // u_f: BSPAI_FP32 or BSPAI_FP16
    float* resid = nullptr;    // ||sbar_k||_2 per column of M'
    int8_t* step_added = nullptr;  // adaptive build: the pass that added each entry (CSR order)
    int32_t* col_info = nullptr;   // adaptive build: solves | conv << 8 | rankdef << 9 | capped << 10
};

struct bspai_bucketed {
    uint32_t magic;
    cudaStream_t stream;
    int32_t n;
    int64_t nnz;
    int32_t q;
    int32_t precs[8];
    bspai::Sell b[8];          // one SELL structure per bucket
    void* val[8] = {nullptr};
    float scale[8];
    float* colscale = nullptr; // per column (e4m3 bucket)
    float* rowscale = nullptr; // per row (e4m3 bucket of a transposed M)
    float* sscale[8] = {nullptr}; // per 32-row slice (fp16 buckets of a batch of systems)
    int64_t nnz_k[8];
    int32_t maxw[8];           // widest slice per bucket (slots per row)
    // copy of M's structure for exporting in CSR order
    bspai::Sell msell;
    int32_t* mrowlen = nullptr;
    int32_t* mcsr_row_ptr = nullptr;
    int8_t* id_sell = nullptr; // bucket id per slot of msell
    bspai::BMDev dev() const;
};

namespace bspai {

// ------------------------------------------------------------------ helpers
int scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t count, cudaStream_t s);
int sell_from_csr(int n, const int32_t* row_ptr, const int32_t* col, const double* val,
                  Sell* out, double** val64, float** val32, int32_t** rowlen, cudaStream_t s);
// packed copy of a plain SELL structure with fp32 values (16-bit columns when they fit)
int sell_packed_copy(const Sell& S, const float* val, Sell* out, float** pval, cudaStream_t s);
// the view A v in u_p reads: the packed copy for fp32, the plain fp64 values for fp64
BMDev up_view(const bspai_matrix* A, int up);
void sell_free(Sell* S, cudaStream_t s);

// launches (defined in spmv.cu)
int launch_bspmv(const BMDev& M, const void* x, int x_prec, void* y, int y_prec, cudaStream_t s);
int launch_bspmv_idx(const BMDev& M, const void* x, int x_prec, void* y, int y_prec, const int* jd,
                     int64_t ldx, int64_t ldy, int yoff, cudaStream_t s);
BMDev single_bucket_view(const Sell& S, const void* val, int prec);
// x0 = M b with the unbucketed M in its u_f (fp32 or fp16 arithmetic), y in fp64
int launch_apply_uf(const bspai_spai* M, const double* x, double* y, cudaStream_t s);
int stage_timeout_take(cudaStream_t s);  // BSPAI_TIMEOUT if a staged SpMV gave up waiting

// defined in matrix.cu
int matrix_create(const bspai_csr_t* A, cudaStream_t s, bspai_matrix** out);
int launch_residual(const bspai_matrix* A, const double* x, const double* b, double* r, double* norms,
                    cudaStream_t s);
int validate_csr(const bspai_csr_t* A, bool need_val, const char* who, cudaStream_t s);
double unit_roundoff(int prec);

// ------------------------------------------------------------------ profiling
bool prof_enabled();
void prof_begin(int cls, cudaStream_t s);
void prof_end(int cls, cudaStream_t s);
struct ProfScope {
    int cls;
    cudaStream_t s;
    bool on;
    ProfScope(int c, cudaStream_t st) : cls(c), s(st), on(prof_enabled()) {
        if (on) prof_begin(cls, s);
    }
    ~ProfScope() {
        if (on) prof_end(cls, s);
    }
};

int num_sms();
// Blocks for a grid-stride loop over n items with bd threads per block: one
// resident wave (per_sm blocks on every SM) at most, so that per-block
// epilogues (one atomic per block) stay few.
inline unsigned wave_grid(int64_t n, int bd = 256, int per_sm = 8) {
    const int64_t need = (n + bd - 1) / bd;
    const int64_t cap = (int64_t)num_sms() * per_sm;
    return (unsigned)(need < cap ? (need > 0 ? need : 1) : cap);
}
void note_launch();  // counts kernel launches (reported by bspai_launch_count)
void count_launches(bool on);  // this thread's launches are (not) counted, e.g. during graph capture

__host__ __device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ------------------------------------------------------------------ device
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Arithmetic in u_f: fp32 (H = false) or fp16 (H = true), values held in fp32
// registers.  An fp16 operation is the correctly rounded fp32 operation
// rounded once more to fp16 (RN-even, fp16's own range with subnormals and
// overflow to Inf).  fp32 carries 24 >= 2 * 11 + 2 significand bits, so by
// Figueroa's double-rounding theorem that is the correctly rounded fp16
// result of +, -, *, / and sqrt: each step is an fp16 operation.
template <bool H>
struct UfOps {
    static __device__ __forceinline__ float r(float x) {
        if constexpr (H) return __half2float(__float2half_rn(x));
        else return x;
    }
    static __device__ __forceinline__ float add(float a, float b) { return r(__fadd_rn(a, b)); }
    static __device__ __forceinline__ float sub(float a, float b) { return r(__fsub_rn(a, b)); }
    static __device__ __forceinline__ float mul(float a, float b) { return r(__fmul_rn(a, b)); }
    static __device__ __forceinline__ float div(float a, float b) { return r(__fdiv_rn(a, b)); }
    static __device__ __forceinline__ float sqrt(float a) { return r(__fsqrt_rn(a)); }
    // an fp64 value rounded once to u_f
    static __device__ __forceinline__ float from64(double x) {
        if constexpr (H) return __half2float(__double2half(x));
        else return __double2float_rn(x);
    }
    // butterfly warp sum with every addition in u_f
    static __device__ __forceinline__ float wsum(float v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = add(v, __shfl_xor_sync(0xffffffffu, v, o));
        return v;
    }
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// atomic max of a non-negative double (bit patterns of non-negative doubles
// order like their values)
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}
// max over the warp of a non-negative double (or NaN) by its bit pattern, the
// order atomic_max_nonneg uses, so the warp's maximum then one atomic per warp
// stores exactly what one atomic per thread would
__device__ __forceinline__ double warp_max_bits(double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, b, o);
        b = t > b ? t : b;
    }
    return __longlong_as_double((long long)b);
}
__device__ __forceinline__ void atomic_max_nonneg(float* addr, float v) {
    atomicMax(reinterpret_cast<unsigned*>(addr), __float_as_uint(v));
}

// One value per warp (read from lane 0) combined across the block by `op`
// (associative and commutative: max, min, integer add), valid in thread 0.
// Every thread of the block calls it; s: blockDim.x / 32 slots of shared
// memory that the caller does not touch between calls.
template <typename T, typename Op>
__device__ __forceinline__ T block_combine(T v, T ident, T* s, Op op) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) s[w] = v;
    __syncthreads();
    T t = ident;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = op(t, s[i]);
    return t;
}

// Values already reduced over each warp (read from lane 0) combined across the
// block by bit pattern, then one atomic_max_nonneg per block and address: the
// same result as one atomic per warp, without a global atomic from every warp
// on one address.  Every thread of the block calls it at the same point
// (blockDim.x a multiple of 32); use it once per kernel.
__device__ __forceinline__ void block_atomic_max_nonneg2(double* a0, double w0, double* a1, double w1) {
    __shared__ unsigned long long s_bm[2][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        s_bm[0][w] = (unsigned long long)__double_as_longlong(w0);
        s_bm[1][w] = (unsigned long long)__double_as_longlong(w1);
    }
    __syncthreads();
    if (w == 0) {
        const bool have = lane < (int)(blockDim.x >> 5);
        unsigned long long b0 = have ? s_bm[0][lane] : 0ull, b1 = have ? s_bm[1][lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t0 = __shfl_xor_sync(0xffffffffu, b0, o);
            const unsigned long long t1 = __shfl_xor_sync(0xffffffffu, b1, o);
            b0 = t0 > b0 ? t0 : b0;
            b1 = t1 > b1 ? t1 : b1;
        }
        if (lane == 0) {
            if (b0) atomicMax(reinterpret_cast<unsigned long long*>(a0), b0);
            if (b1) atomicMax(reinterpret_cast<unsigned long long*>(a1), b1);
        }
    }
}
__device__ __forceinline__ void block_atomic_max_nonneg(double* a0, double w0) {
    __shared__ unsigned long long s_bm1[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) s_bm1[w] = (unsigned long long)__double_as_longlong(w0);
    __syncthreads();
    if (w == 0) {
        unsigned long long b0 = lane < (int)(blockDim.x >> 5) ? s_bm1[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t0 = __shfl_xor_sync(0xffffffffu, b0, o);
            b0 = t0 > b0 ? t0 : b0;
        }
        if (lane == 0 && b0) atomicMax(reinterpret_cast<unsigned long long*>(a0), b0);
    }
}

// Grid-wide barrier for cooperative launches (all blocks co-resident).
// Generation counting: the last block to arrive resets the counter and bumps
// the generation; the others wait for the bump.  Every wait is bounded by
// `timeout_ns` of %globaltimer; on expiry the block sets bar->err and every
// waiter returns false, so the kernel can exit and the host can report
// BSPAI_TIMEOUT (and must reset the barrier before reusing it).
struct GridBar {
    unsigned count;
    unsigned gen;
    int err;
    unsigned seq;  // tagged-slot reductions completed on this state (k_mgs_res)
};

__device__ __forceinline__ bool grid_sync(GridBar* bar, unsigned long long timeout_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned nb = gridDim.x;
        unsigned gen = ld_acquire_u32(&bar->gen);
        __threadfence();
        unsigned arrived = atomicAdd(&bar->count, 1u);
        if (arrived == nb - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            unsigned long long t0 = globaltimer_ns();
            while (ld_acquire_u32(&bar->gen) == gen) {
                if (*(volatile int*)&bar->err) { ok = 0; break; }
                if (globaltimer_ns() - t0 > timeout_ns) {
                    atomicExch(&bar->err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (*(volatile int*)&bar->err) ok = 0;
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace bspai
