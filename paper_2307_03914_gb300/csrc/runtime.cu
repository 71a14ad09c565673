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
// = total), one CTA: each thread sums a contiguous chunk, the chunk sums are
// scanned across the block, then each thread writes its chunk.
__global__ void k_scan_i64(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t count) {
    constexpr int T = 1024;
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t s_carry;
    const int tid = threadIdx.x;
    int64_t chunk = (count + T - 1) / T;
    int64_t lo = (int64_t)tid * chunk;
    int64_t hi = lo + chunk < count ? lo + chunk : count;
    int64_t sum = 0;
    for (int64_t i = lo; i < hi; ++i) sum += in[i];
    // block-wide exclusive scan of the chunk sums
    int lane = tid & 31, w = tid >> 5;
    int64_t v = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_tot[w] = v;
    __syncthreads();
    if (w == 0) {
        int64_t t = warp_tot[lane];
        int64_t u = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, u, o);
            if (lane >= o) u += y;
        }
        warp_tot[lane] = u - t;  // exclusive over warps
        if (lane == 31) s_carry = u;
    }
    __syncthreads();
    int64_t run = v - sum + warp_tot[w];
    for (int64_t i = lo; i < hi; ++i) {
        out[i] = run;
        run += in[i];
    }
    if (tid == 0) out[count] = s_carry;
}

int scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t count, cudaStream_t s) {
    k_scan_i64<<<1, 1024, 0, s>>>(in, out, count);
    note_launch();
    CUDA_LAUNCH_CHECK();
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
