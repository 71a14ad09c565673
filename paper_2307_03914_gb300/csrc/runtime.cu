// runtime.cu -- errors, stream-ordered allocation, kernel-class timing, the
// exclusive scan used to lay out SELL slices, and handle release.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace bspai {

static thread_local std::string t_err = "no error";

int set_error(int code, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return code;
}

int cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    const char* f = file;
    for (const char* p = file; *p; ++p)
        if (*p == '/') f = p + 1;
    set_error(e == cudaErrorMemoryAllocation ? BSPAI_ERR_NOMEM : BSPAI_ERR_CUDA, "%s:%d: %s: %s",
              f, line, what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? BSPAI_ERR_NOMEM : BSPAI_ERR_CUDA;
}

static std::atomic<long long> g_launches{0};
static thread_local bool t_count_on = true;
void count_launches(bool on) { t_count_on = on; }
void note_launch() {
    if (t_count_on) g_launches.fetch_add(1, std::memory_order_relaxed);
}

static std::once_flag g_pool_once;

int dalloc(void** p, size_t bytes, cudaStream_t s) {
    std::call_once(g_pool_once, [] {
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
    }
    return BSPAI_OK;
}

void dfree(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// ------------------------------------------------------------------ profiling
namespace {
struct ProfRec {
    int cls;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_pending;
std::vector<cudaEvent_t> g_event_pool;
double g_prof_ms[BSPAI_K_COUNT];
int64_t g_prof_n[BSPAI_K_COUNT];

cudaEvent_t take_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}
thread_local std::vector<ProfRec> t_open;
}  // namespace

bool prof_enabled() { return g_prof_on; }

void prof_begin(int cls, cudaStream_t s) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    ProfRec r{cls, take_event(), take_event()};
    cudaEventRecord(r.a, s);
    t_open.push_back(r);
}

void prof_end(int cls, cudaStream_t s) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    if (t_open.empty()) return;
    ProfRec r = t_open.back();
    t_open.pop_back();
    (void)cls;
    cudaEventRecord(r.b, s);
    g_prof_pending.push_back(r);
}

// ------------------------------------------------------------------ scan
// Exclusive prefix sum of `count` int64 values into out[0..count] (out[count]
// = total).  Tiles of kScanTile values, one block each, in two launches:
// k_scan_sums adds every tile, k_scan_apply gives each tile the sum of the
// tiles before it plus its own exclusive scan.  Every global access is
// coalesced (the tile is staged in shared memory, where each thread takes
// kScanK consecutive values).  Integer sums: the result does not depend on
// the order of the additions.
constexpr int kScanT = 256, kScanK = 8, kScanTile = kScanT * kScanK;

__device__ __forceinline__ int64_t block_sum_i64(int64_t v, int64_t* s_w) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();  // s_w may still be read by an earlier call
    if (lane == 0) s_w[w] = v;
    __syncthreads();
    int64_t t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s_w[i];
    return t;
}

__global__ void __launch_bounds__(kScanT) k_scan_sums(const int64_t* __restrict__ in, int64_t count,
                                                      int64_t* __restrict__ tsum) {
    __shared__ int64_t s_w[kScanT / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t v = 0;
#pragma unroll
    for (int k = 0; k < kScanK; ++k) {
        const int64_t i = base + k * kScanT + threadIdx.x;
        if (i < count) v += in[i];
    }
    v = block_sum_i64(v, s_w);
    if (threadIdx.x == 0) tsum[blockIdx.x] = v;
}

__global__ void __launch_bounds__(kScanT) k_scan_apply(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                                                       int64_t count, const int64_t* __restrict__ tsum) {
    __shared__ int64_t tile[kScanTile];
    __shared__ int64_t s_w[kScanT / 32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    // the tiles before this one
    int64_t off = 0;
    for (int t = tid; t < (int)blockIdx.x; t += kScanT) off += tsum[t];
    off = block_sum_i64(off, s_w);
#pragma unroll
    for (int k = 0; k < kScanK; ++k) {
        const int64_t i = base + k * kScanT + tid;
        tile[k * kScanT + tid] = i < count ? in[i] : 0;
    }
    __syncthreads();
    int64_t loc[kScanK];
    int64_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanK; ++k) {
        loc[k] = tile[tid * kScanK + k];
        sum += loc[k];
    }
    // exclusive scan of the thread sums across the block
    int64_t v = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    __syncthreads();  // s_w was last read in block_sum_i64
    if (lane == 31) s_w[w] = v;
    __syncthreads();
    int64_t before = 0;
    for (int i = 0; i < w; ++i) before += s_w[i];
    int64_t run = off + before + v - sum;
#pragma unroll
    for (int k = 0; k < kScanK; ++k) {
        tile[tid * kScanK + k] = run;
        run += loc[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanK; ++k) {
        const int64_t i = base + k * kScanT + tid;
        if (i < count) out[i] = tile[k * kScanT + tid];
    }
    if (blockIdx.x == gridDim.x - 1 && tid == kScanT - 1) out[count] = run;
}

int scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t count, cudaStream_t s) {
    if (count <= 0) {
        CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return BSPAI_OK;
    }
    const int64_t tiles = ceil_div(count, (int64_t)kScanTile);
    if (tiles > INT32_MAX) return set_error(BSPAI_ERR_UNSUPPORTED, "scan of %lld values", (long long)count);
    int64_t* tsum = nullptr;
    BSPAI_TRY(dalloc_t(&tsum, (size_t)tiles, s));
    k_scan_sums<<<(unsigned)tiles, kScanT, 0, s>>>(in, count, tsum);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_scan_apply<<<(unsigned)tiles, kScanT, 0, s>>>(in, out, count, tsum);
        note_launch();
        e = cudaGetLastError();
    }
    dfree(tsum, s);
    if (e != cudaSuccess) return cuda_error(e, "k_scan", __FILE__, __LINE__);
    return BSPAI_OK;
}

void sell_free(Sell* S, cudaStream_t s) {
    dfree(S->sptr, s);
    dfree(S->col, s);
    dfree(S->col16, s);
    S->sptr = nullptr;
    S->col = nullptr;
    S->col16 = nullptr;
}

}  // namespace bspai

using namespace bspai;

extern "C" {

const char* bspai_last_error(void) { return t_err.c_str(); }

int bspai_version(void) { return 10000 * 0 + 100 * 1 + 0; }

long long bspai_launch_count(void) { return g_launches.load(); }

void bspai_opts_default(bspai_opts_t* o) {
    if (!o) return;
    o->tau = 1e-4;
    o->kmax = 0;
    o->i_max = 0;
    o->x0_given = 0;
    o->max_blocks = 0;
    o->u_stop = 0.0;
    o->stagnation = 0.0;
    o->barrier_timeout_s = 0.0;
    o->basis_bytes_max = 0;
}

int bspai_profile_enable(int on) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof_on = on != 0;
    return BSPAI_OK;
}

int bspai_profile_read(bspai_profile_t* out, int reset) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    for (auto& r : g_prof_pending) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) return cuda_error(e, "profile event", __FILE__, __LINE__);
        g_prof_ms[r.cls] += ms;
        g_prof_n[r.cls] += 1;
        g_event_pool.push_back(r.a);
        g_event_pool.push_back(r.b);
    }
    g_prof_pending.clear();
    if (out) {
        for (int c = 0; c < BSPAI_K_COUNT; ++c) {
            out->ms[c] = g_prof_ms[c];
            out->launches[c] = g_prof_n[c];
        }
    }
    if (reset) {
        for (int c = 0; c < BSPAI_K_COUNT; ++c) {
            g_prof_ms[c] = 0.0;
            g_prof_n[c] = 0;
        }
    }
    return BSPAI_OK;
}

int bspai_free(void* h) {
    if (!h) return BSPAI_OK;
    uint32_t magic = *reinterpret_cast<uint32_t*>(h);
    if (magic == kMagicA) {
        auto* A = reinterpret_cast<bspai_matrix*>(h);
        cudaStream_t s = A->stream;
        sell_free(&A->sell, s);
        sell_free(&A->psell, s);
        dfree(A->val64, s);
        dfree(A->val32, s);
        dfree(A->pval32, s);
        dfree(A->norm_inf, s);
        dfree(A->rowlen, s);
        dfree(A->csr_row_ptr, s);
        A->magic = kMagicDead;
        delete A;
    } else if (magic == kMagicM) {
        auto* M = reinterpret_cast<bspai_spai*>(h);
        cudaStream_t s = M->stream;
        sell_free(&M->sell, s);
        dfree(M->rowlen, s);
        dfree(M->csr_row_ptr, s);
        dfree(M->val, s);
        dfree(M->resid, s);
        dfree(M->step_added, s);
        dfree(M->col_info, s);
        M->magic = kMagicDead;
        delete M;
    } else if (magic == kMagicBM) {
        auto* B = reinterpret_cast<bspai_bucketed*>(h);
        cudaStream_t s = B->stream;
        for (int k = 0; k < B->q; ++k) {
            sell_free(&B->b[k], s);
            dfree(B->val[k], s);
            dfree(B->sscale[k], s);
        }
        dfree(B->colscale, s);
        dfree(B->rowscale, s);
        sell_free(&B->msell, s);
        dfree(B->mrowlen, s);
        dfree(B->mcsr_row_ptr, s);
        dfree(B->id_sell, s);
        B->magic = kMagicDead;
        delete B;
    } else {
        return set_error(BSPAI_ERR_INVALID, "bspai_free: not a live bspai handle");
    }
    return BSPAI_OK;
}

}  // extern "C"
