// gmres.cu -- left-preconditioned MGS-GMRES and the refinement loop of Alg 3.1.
//
// Per Arnoldi step j (the "hot loop" of the method) three launches run on the
// solve's stream, with no host synchronisation between steps:
//   w = A v_j               (u_p, SELL SpMV)                       spmv.cu
//   z = M w -> V(:, j+1)    (Alg 2.3 bucketed SpMV, stored in u_g) spmv.cu
//   k_mgs                   (cooperative, persistent)              this file
// The Krylov index j and the "done" flag live in device memory (GmresState);
// every kernel of a step reads them, so the host enqueues steps in chunks and
// only reads the flag between chunks.  Steps enqueued after convergence
// return immediately.
//
// k_mgs keeps one contiguous range of rows per block.  Modified Gram-Schmidt
// needs the j+1 dot products in sequence; pass i fuses the update by the
// previous coefficient with the next dot product, z <- z - h_{i-1} v_{i-1};
// partial += v_i . z, so each basis vector is streamed once per step.  The
// block partial sums go to a global array, one grid barrier, and every block
// then adds the partials in the same fixed order, so all blocks hold the same
// h_ij (deterministic, no atomics).  The last pass forms ||z||_2 and
// normalises v_{j+1}; block 0 then applies the Givens rotations (fp64) and
// tests |g_{j+1}| <= tau ||M r||_2.  j + 2 barriers per step, each bounded in
// time (BSPAI_TIMEOUT).
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "tags.cuh"

namespace bspai {

struct GmresState {
    int j;        // completed Arnoldi steps (= k)
    int done;     // 1 once converged, broken down, failed or at kmax
    int status;   // BSPAI_OK, BSPAI_TIMEOUT, BSPAI_NONFINITE
    int kmax;
    double beta;  // ||M r||_2 (in u_g)
    double tau;
    double target;  // > 0: stop at |g| <= target instead of the tau test (restarted cycles)
    double res;   // |g_k|
    double hlast;
    GridBar bar;
};

template <typename T>
struct Ar;
template <>
struct Ar<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float sqrt(float a) { return __fsqrt_rn(a); }
    static __device__ __forceinline__ float from(double a) { return __double2float_rn(a); }
};
template <>
struct Ar<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double sqrt(double a) { return __dsqrt_rn(a); }
    static __device__ __forceinline__ double from(double a) { return a; }
};

__global__ void k_state_init(GmresState* st, int kmax, double tau, double target) {
    st->j = 0;
    st->done = 0;
    st->status = BSPAI_OK;
    st->kmax = kmax;
    st->beta = 0.0;
    st->tau = tau;
    st->target = target;
    st->res = 0.0;
    st->hlast = 0.0;
    st->bar.count = 0;
    st->bar.err = 0;
}

__device__ __forceinline__ void block_rows(int n, int G, int64_t& r0, int64_t& r1) {
    int64_t chunk = ceil_div(ceil_div(n, G), 32) * 32;
    r0 = (int64_t)blockIdx.x * chunk;
    r1 = r0 + chunk < n ? r0 + chunk : n;
}
__device__ __forceinline__ void block_rows(int n, int64_t& r0, int64_t& r1) { block_rows(n, (int)gridDim.x, r0, r1); }

// Sum of `v` over the whole grid, identical in every block: block sum in a
// fixed tree, partials to part[slot*G + block], barrier, then every block adds
// the G partials in the same order.  `ok` is false if the barrier failed.
template <typename T>
__device__ __forceinline__ T grid_sum(T v, T* part, int slot, GridBar* bar, unsigned long long tmo, bool& ok) {
    __shared__ T s_w[32];
    __shared__ T s_tot;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    if (lane == 0) s_w[w] = v;
    __syncthreads();
    if (w == 0) {
        T t = lane < nw ? s_w[lane] : T(0);
        t = warp_sum(t);
        if (lane == 0) part[(int64_t)slot * gridDim.x + blockIdx.x] = t;
    }
    ok = grid_sync(bar, tmo);
    if (!ok) return T(0);
    if (w == 0) {
        T t = T(0);
        for (int b = lane; b < (int)gridDim.x; b += 32)
            t = Ar<T>::add(t, *(volatile T*)&part[(int64_t)slot * gridDim.x + b]);
        t = warp_sum(t);
        if (lane == 0) s_tot = t;
    }
    __syncthreads();
    return s_tot;
}

// beta = ||s||_2 of V(:, 0) = s = M r, then v_0 = s / beta and g_0 = beta
template <typename T>
__global__ void __launch_bounds__(512) k_gmres_start(T* __restrict__ V, int n, GmresState* st, double* g, T* part,
                                                     unsigned long long tmo) {
    int64_t r0, r1;
    block_rows(n, r0, r1);
    T acc = T(0);
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) acc = Ar<T>::add(acc, Ar<T>::mul(V[r], V[r]));
    bool ok;
    const T tot = grid_sum(acc, part, 0, &st->bar, tmo, ok);
    if (!ok) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->status = BSPAI_TIMEOUT;
            st->done = 1;
        }
        return;
    }
    const T beta = Ar<T>::sqrt(tot);
    const bool fin = isfinite((double)beta);
    if (beta > T(0) && fin)
        for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) V[r] = Ar<T>::div(V[r], beta);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->beta = (double)beta;
        st->res = (double)beta;
        g[0] = (double)beta;
        st->done = !(beta > T(0)) || !fin;
        if (!fin) st->status = BSPAI_NONFINITE;
    }
}

// The new rotation of step j from the swept column (hc[j] = carry, the entry the
// earlier rotations handed on, hc[j+1] = hn = h_{j+1,j}), the update of g and
// the tau test (fp64)
__device__ void givens_finish(int j, int kmax, double hn, double carry, double* __restrict__ hc, double* cs,
                              double* sn, double* g, GmresState* st) {
    hc[j] = carry;
    hc[j + 1] = hn;
    const double a = carry, b = hn;
    const double rr = __dsqrt_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)));
    double c = 1.0, s = 0.0;
    if (rr != 0.0) {
        c = __ddiv_rn(a, rr);
        s = __ddiv_rn(b, rr);
    }
    cs[j] = c;
    sn[j] = s;
    hc[j] = rr;
    hc[j + 1] = 0.0;
    g[j + 1] = __dmul_rn(-s, g[j]);
    g[j] = __dmul_rn(c, g[j]);
    const double res = fabs(g[j + 1]);
    const int k = j + 1;
    const bool fin = isfinite(res) && isfinite(hn) && isfinite(rr);
    st->res = res;
    st->hlast = hn;
    st->j = k;
    if (!fin) st->status = BSPAI_NONFINITE;
    const double lvl = st->target > 0.0 ? st->target : __dmul_rn(st->tau, st->beta);
    st->done = (res <= lvl) || hn == 0.0 || k >= kmax || !fin;
}

// rotation i of the earlier steps applied to the pair (carry, h_{i+1,j}): the
// rotated h_{i,j} is returned, the entry handed on to rotation i + 1 stays in carry
__device__ __forceinline__ double givens_apply(double ci, double si, double& carry, double hi1) {
    const double t1 = __dadd_rn(__dmul_rn(ci, carry), __dmul_rn(si, hi1));
    carry = __dadd_rn(__dmul_rn(-si, carry), __dmul_rn(ci, hi1));
    return t1;
}

// Givens rotations on column j of H (written unrotated), update of g and the tau test (fp64)
__device__ void givens_step(int j, int kmax, double hn, double* H, double* cs, double* sn, double* g,
                            GmresState* st) {
    double* __restrict__ hc = H + (int64_t)j * (kmax + 1);
    const double* __restrict__ c_ = cs;
    const double* __restrict__ s_ = sn;
    // the previous rotations applied to the new column; the entry each rotation hands
    // to the next stays in a register, so only the running value is a dependent chain
    // (the stored coefficients and column entries are independent loads)
    double carry = hc[0];
    for (int i = 0; i < j; ++i) hc[i] = givens_apply(c_[i], s_[i], carry, hc[i + 1]);
    givens_finish(j, kmax, hn, carry, hc, cs, sn, g, st);
}

template <typename T>
__global__ void __launch_bounds__(512) k_mgs(T* __restrict__ V, int64_t ldv, int n, GmresState* st, double* H,
                                             double* cs, double* sn, double* g, T* part, unsigned long long tmo) {
    __shared__ int s_j, s_done, s_kmax;
    if (threadIdx.x == 0) {
        s_j = st->j;
        s_done = st->done;
        s_kmax = st->kmax;
    }
    __syncthreads();
    if (s_done) return;
    const int j = s_j, kmax = s_kmax;
    int64_t r0, r1;
    block_rows(n, r0, r1);
    T* z = V + (int64_t)(j + 1) * ldv;
    T hprev = T(0);
    for (int i = 0; i <= j + 1; ++i) {
        const T* vi = V + (int64_t)(i <= j ? i : j) * ldv;
        const T* vp = V + (int64_t)(i > 0 ? i - 1 : 0) * ldv;
        T acc = T(0);
        if (i == 0) {
            for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x)
                acc = Ar<T>::add(acc, Ar<T>::mul(vi[r], z[r]));
        } else if (i <= j) {
            for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
                const T zr = Ar<T>::sub(z[r], Ar<T>::mul(hprev, vp[r]));
                z[r] = zr;
                acc = Ar<T>::add(acc, Ar<T>::mul(vi[r], zr));
            }
        } else {
            for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
                const T zr = Ar<T>::sub(z[r], Ar<T>::mul(hprev, vp[r]));
                z[r] = zr;
                acc = Ar<T>::add(acc, Ar<T>::mul(zr, zr));
            }
        }
        bool ok;
        const T h = grid_sum(acc, part, i & 1, &st->bar, tmo, ok);
        if (!ok) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                st->status = BSPAI_TIMEOUT;
                st->done = 1;
            }
            return;
        }
        if (i <= j) {
            if (blockIdx.x == 0 && threadIdx.x == 0) H[(int64_t)j * (kmax + 1) + i] = (double)h;
            hprev = h;
        } else {
            const T hn = Ar<T>::sqrt(h);
            if (hn > T(0) && isfinite((double)hn))
                for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) z[r] = Ar<T>::div(z[r], hn);
            if (blockIdx.x == 0 && threadIdx.x == 0) givens_step(j, kmax, (double)hn, H, cs, sn, g, st);
        }
    }
}

constexpr int kMgsBlocks = 64;  // fewest blocks the on-chip MGS kernel is given
// A block's bytes of one basis vector (at the instance's capacity) from which
// an on-chip MGS instance polls its reductions by bulk copies
// (tag_poll_warp_bulk) instead of loads.  Measured (fp32, 64-128 blocks,
// 64-step GMRES runs): load polling 5 % faster at 4 KB per block
// (n = 64,000), even at 7 KB; bulk polling 11 / 3 / 4 % faster at 16 / 32 /
// 64 KB (n = 262,144 / 512,000 / 2,097,152); with 9 blocks per solve (16
// right-hand sides side by side) and 29 KB per block, slower.  Instances whose
// capacity is below the threshold are compiled without the bulk path (their
// load poll's code unchanged); the others take it when the launch asks.
constexpr int64_t kBulkPollBytes = 16 * 1024;

// The Givens block: with giv = 1 the last block of an on-chip MGS launch takes
// no rows.  Its first warp reads every pass's total from the same tagged slots
// as the other blocks (so the same values), applies rotation i - 1 of the
// earlier steps to column j as soon as h_{i,j} has arrived -- while the other
// blocks run the later passes -- and after the last pass forms the new
// rotation, g and the tau test.  One thread's sweep over the earlier
// rotations costs about 480 cycles per rotation on GB300's narrow fp64 pipe
// (21 us at j = 90), and here it overlaps the passes instead of following the
// last one.  Same operations in the same order as givens_step.
template <typename T>
__device__ void givens_block(int j, int kmax, double* H, double* cs, double* sn, double* g, GmresState* st,
                             const unsigned long long* tags, int G, unsigned seq0, unsigned long long tmo) {
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    double* __restrict__ hc = H + (int64_t)j * (kmax + 1);
    double carry = 0.0;
    T hz = T(0);
    bool ok = true;
    for (int i = 1; i <= j + 2; ++i) {
        T h;
        if (!tag_poll_warp<T>(tags, (i - 1) & 1, seq0 + (unsigned)i, G, &st->bar, tmo, &h)) {
            ok = false;
            break;
        }
        if (i == j + 2) {
            hz = h;
            break;
        }
        const int r = i - 1;  // h = h_{r,j}
        if (lane == 0) {
            if (r == 0) carry = (double)h;
            else hc[r - 1] = givens_apply(cs[r - 1], sn[r - 1], carry, (double)h);
        }
    }
    if (lane != 0) return;
    if (!ok) {
        st->status = BSPAI_TIMEOUT;
        st->done = 1;
        return;
    }
    // every block has read seq0 before its last partial, and this block read it
    // at its start: advance it for the next launch
    st->bar.seq = seq0 + (unsigned)j + 2u;
    givens_finish(j, kmax, (double)Ar<T>::sqrt(hz), carry, hc, cs, sn, g, st);
}

// MGS step with the new vector z resident on chip: one block per SM owns a
// contiguous range of rows, holds z for them in shared memory for all j + 2
// passes, and streams each basis vector v_i exactly once (R rows per thread
// of a BD-thread block, all loads of a pass issued before the thread waits on
// the previous pass's reduction; BD = 512 for many rows per block, so that
// the 2 R values a thread keeps stay in registers).  Per pass i: z <- z - h_{i-1} v_{i-1} (v_{i-1} kept in registers),
// partial += v_i . z, arrive; the last pass forms ||z||_2 and writes v_{j+1}.
// Same arithmetic as k_mgs (fp32 or fp64, no fused multiply-add).
template <typename T, int R, int BD>
__global__ void __launch_bounds__(BD, 1) k_mgs_res(T* __restrict__ V, int64_t ldv, int n, GmresState* st,
                                                     double* H, double* cs, double* sn, double* g,
                                                     unsigned long long* tags, unsigned long long tmo, int giv,
                                                     int bulk) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T* zs = reinterpret_cast<T*>(smraw);
    constexpr bool kBulk = (int64_t)R * BD * (int64_t)sizeof(T) >= kBulkPollBytes;  // and bulk: the launch's choice
    __shared__ T s_w[32];
    __shared__ T s_tot;
    __shared__ unsigned s_seq;
    __shared__ int s_ok, s_j, s_done, s_kmax;
    __shared__ __align__(16) unsigned long long s_slots[kBulk ? 2 * kTagMaxBlocks + 2 : 2];  // warp 0's copies
    __shared__ __align__(8) uint64_t s_mbar;
    unsigned phase = 0;
    if (threadIdx.x == 0) {
        s_j = st->j;
        s_done = st->done;
        s_kmax = st->kmax;
        s_seq = *(volatile unsigned*)&st->bar.seq;  // reductions of this launch are s_seq + 1, s_seq + 2, ...
        if (kBulk) {
            mbar_init(&s_mbar, 1);
            mbar_init_fence();
        }
    }
    __syncthreads();
    if (s_done) return;
    const int j = s_j, kmax = s_kmax;
    const unsigned seq0 = s_seq;
    const int G = gridDim.x - giv;  // blocks that hold rows and publish partial sums
    if (giv && blockIdx.x == G) {
        givens_block<T>(j, kmax, H, cs, sn, g, st, tags, G, seq0, tmo);
        return;
    }
    int64_t r0, r1;
    block_rows(n, G, r0, r1);
    const int nb = r1 > r0 ? (int)(r1 - r0) : 0;
    const int tid = threadIdx.x;
    constexpr int bd = BD;
    T* z = V + (int64_t)(j + 1) * ldv + r0;
    const T* v0 = V + r0;
    T vcur[R], vnext[R];
#pragma unroll
    for (int t = 0; t < R; ++t) {
        const int lr = tid + t * bd;
        vcur[t] = T(0);
        vnext[t] = T(0);
        if (lr < nb) {
            zs[lr] = z[lr];
            vcur[t] = v0[lr];
        }
    }
    T acc = T(0);
#pragma unroll
    for (int t = 0; t < R; ++t) {
        const int lr = tid + t * bd;
        if (lr < nb) acc = Ar<T>::add(acc, Ar<T>::mul(vcur[t], zs[lr]));
    }
    tag_arrive(acc, tags, 0, seq0 + 1u, s_w, G);
    for (int i = 1; i <= j + 1; ++i) {
        if (i <= j) {
            const T* vi = V + (int64_t)i * ldv + r0;
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int lr = tid + t * bd;
                if (lr < nb) vnext[t] = vi[lr];
            }
        }
        const T h = tag_wait_bulk(tags, (i - 1) & 1, seq0 + (unsigned)i, &st->bar, tmo, &s_tot, &s_ok, G, s_slots,
                                  &s_mbar, phase, kBulk && bulk);
        if (!s_ok) {
            if (blockIdx.x == 0 && tid == 0) {
                st->status = BSPAI_TIMEOUT;
                st->done = 1;
            }
            return;
        }
        if (!giv && blockIdx.x == 0 && tid == 0) H[(int64_t)j * (kmax + 1) + (i - 1)] = (double)h;
        acc = T(0);
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int lr = tid + t * bd;
            if (lr < nb) {
                const T zr = Ar<T>::sub(zs[lr], Ar<T>::mul(h, vcur[t]));
                zs[lr] = zr;
                acc = Ar<T>::add(acc, Ar<T>::mul(i <= j ? vnext[t] : zr, zr));
            }
        }
        tag_arrive(acc, tags, i & 1, seq0 + (unsigned)i + 1u, s_w, G);
#pragma unroll
        for (int t = 0; t < R; ++t) vcur[t] = vnext[t];
    }
    const T h2 = tag_wait_bulk(tags, (j + 1) & 1, seq0 + (unsigned)j + 2u, &st->bar, tmo, &s_tot, &s_ok, G, s_slots,
                               &s_mbar, phase, kBulk && bulk);
    if (!s_ok) {
        if (blockIdx.x == 0 && tid == 0) {
            st->status = BSPAI_TIMEOUT;
            st->done = 1;
        }
        return;
    }
    // every block has read seq0 (its first slot carries seq0 + 1): advance it
    // (with a Givens block, that block advances it: it may have started last)
    if (!giv && blockIdx.x == 0 && tid == 0) st->bar.seq = seq0 + (unsigned)j + 2u;
    const T hn = Ar<T>::sqrt(h2);
    const bool norm = hn > T(0) && isfinite((double)hn);
#pragma unroll
    for (int t = 0; t < R; ++t) {
        const int lr = tid + t * bd;
        if (lr < nb) z[lr] = norm ? Ar<T>::div(zs[lr], hn) : zs[lr];
    }
    if (!giv && blockIdx.x == 0 && tid == 0) givens_step(j, kmax, (double)hn, H, cs, sn, g, st);
}

// y = R^-1 g by column-oriented back substitution (fp64): for i = k-1 .. 0,
// y_i = g_i / R_ii and g_t -= R_ti y_i for t < i (each g_t sees the same
// operations in the same order as a plain column back substitution).  When
// g and the triangle of R fit in kBackSmem bytes, the block first copies them
// into shared memory with every load in flight at once, and warp 0 then runs
// the k dependent rows from there.  Otherwise the whole block runs the rows:
// thread x holds rows x + kBackThreads c of the current column in registers
// and loads the next column's while the current row is processed, the owner
// of row i divides, and one barrier per row hands y_i to the others.
// Launch: one block of kBackThreads, kBackSmem bytes of dynamic shared memory.
constexpr int kBackThreads = 512;
constexpr size_t kBackSmem = 47 * 1024;  // with the static s_y, within the 48 KB a launch gets without opting in
constexpr int kBackC = 8;  // rows per thread in the streamed form: k <= kBackThreads * kBackC
__global__ void __launch_bounds__(kBackThreads) k_backsolve(const GmresState* st, const double* __restrict__ H,
                                                            const double* __restrict__ g, double* __restrict__ y,
                                                            int kmax) {
    extern __shared__ double sg[];
    __shared__ double s_y[2];
    const int k = st->j;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int t = tid; t < k; t += blockDim.x) sg[t] = g[t];
    if ((size_t)k * (k + 3) / 2 * sizeof(double) <= kBackSmem) {
        // sg[0, k): g; then column i of R (rows 0 .. i) at sg + k + i (i + 1) / 2;
        // warp w copies columns w, w + 16, ... (integer indexing only: the fp64 pipe is narrow)
        double* R = sg + k;
        for (int i = tid >> 5; i < k; i += blockDim.x >> 5) {
            const double* hc = H + (int64_t)i * (kmax + 1);
            double* rc = R + i * (i + 1) / 2;
            for (int t = lane; t <= i; t += 32) rc[t] = hc[t];
        }
        __syncthreads();
        if (tid >= 32) return;
        for (int i = k - 1; i >= 0; --i) {
            const double* rc = R + i * (i + 1) / 2;
            const double yi = __ddiv_rn(sg[i], rc[i]);
            if (lane == 0) y[i] = yi;
            for (int t = lane; t < i; t += 32) sg[t] = __dsub_rn(sg[t], __dmul_rn(rc[t], yi));
            __syncwarp();
        }
        return;
    }
    // rows t = tid + kBackThreads c of column i (t <= i) in registers; g_t stays with its owner
    double nxt[kBackC], cur[kBackC];
    auto fetch = [&](int i) {
        const double* hc = H + (int64_t)i * (kmax + 1);
#pragma unroll
        for (int c = 0; c < kBackC; ++c) {
            const int t = tid + kBackThreads * c;
            nxt[c] = t <= i ? hc[t] : 0.0;
        }
    };
    double gt[kBackC];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kBackC; ++c) {
        const int t = tid + kBackThreads * c;
        gt[c] = t < k ? sg[t] : 0.0;
    }
    if (k > 0) fetch(k - 1);
    for (int i = k - 1; i >= 0; --i) {
#pragma unroll
        for (int c = 0; c < kBackC; ++c) cur[c] = nxt[c];
        if (i > 0) fetch(i - 1);
        if (tid == i % kBackThreads) {
            const int ci = i / kBackThreads;
            double gi = 0.0, di = 1.0;
#pragma unroll
            for (int c = 0; c < kBackC; ++c)
                if (c == ci) {
                    gi = gt[c];
                    di = cur[c];
                }
            const double yi = __ddiv_rn(gi, di);
            s_y[i & 1] = yi;
            y[i] = yi;
        }
        __syncthreads();
        const double yi = s_y[i & 1];
#pragma unroll
        for (int c = 0; c < kBackC; ++c) {
            const int t = tid + kBackThreads * c;
            if (t < i) gt[c] = __dsub_rn(gt[c], __dmul_rn(cur[c], yi));
        }
    }
}

// d = V y in u_g (y rounded to u_g, sequential over j), then x += d in fp64;
// max|d| -> norms[0], max|x| -> norms[1]
template <typename T>
__global__ void __launch_bounds__(256) k_gmres_update(const T* __restrict__ V, int64_t ldv, int n,
                                                      const GmresState* st, const double* __restrict__ y,
                                                      double* __restrict__ x, double* __restrict__ dout,
                                                      double* __restrict__ norms, int u32) {
    extern __shared__ unsigned char sraw[];
    T* sy = reinterpret_cast<T*>(sraw);
    const int k = st->j;
    for (int t = threadIdx.x; t < k; t += blockDim.x) sy[t] = Ar<T>::from(y[t]);
    __syncthreads();
    double dabs = 0.0, xabs = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        // the products added in order of j; the loads of 8 columns issued before their adds
        T acc = T(0);
        int jj = 0;
        for (; jj + 8 <= k; jj += 8) {
            T v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = V[(int64_t)(jj + u) * ldv + r];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc = Ar<T>::add(acc, Ar<T>::mul(v[u], sy[jj + u]));
        }
        for (; jj < k; ++jj) acc = Ar<T>::add(acc, Ar<T>::mul(V[(int64_t)jj * ldv + r], sy[jj]));
        double d = (double)acc;
        // working precision u = fp32: d stored in u, x = fl32(x + d) (x and d
        // are fp32 values, so the fp64 sum rounds to the correctly rounded fp32 sum)
        if (u32) d = (double)__double2float_rn(d);
        if (dout) dout[r] = d;
        double xn = 0.0;
        if (x) {
            xn = __dadd_rn(x[r], d);
            if (u32) xn = (double)__double2float_rn(xn);
            x[r] = xn;
        }
        double da = fabs(d), xa = fabs(xn);
        if (!(da <= 1.7976931348623157e308)) da = __longlong_as_double(0x7ff0000000000000LL);
        if (!(xa <= 1.7976931348623157e308)) xa = __longlong_as_double(0x7ff0000000000000LL);
        dabs = fmax(dabs, da);
        xabs = fmax(xabs, xa);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dabs = fmax(dabs, __shfl_xor_sync(0xffffffffu, dabs, o));
        xabs = fmax(xabs, __shfl_xor_sync(0xffffffffu, xabs, o));
    }
    block_atomic_max_nonneg2(norms, dabs, norms + 1, xabs);
}

__global__ void k_absmax(int n, const double* __restrict__ v, double* __restrict__ out) {
    double a = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double t = fabs(v[r]);
        if (!(t <= 1.7976931348623157e308)) t = __longlong_as_double(0x7ff0000000000000LL);
        a = fmax(a, t);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    block_atomic_max_nonneg(out, a);
}

// k_mgs_res for fp32 with the rows of a thread taken in adjacent pairs: every
// multiply and add is a packed two-lane fp32 operation (each lane correctly
// rounded, no fused multiply-add: the same arithmetic per element), z and the
// basis rows move as float2, and the thread's partial sum is carried in two
// lanes that are added at the end.  z stays in registers for all j + 2 passes
// (2 P values per thread beside v_{i-1} and v_i: at most 128 registers for
// P = 16 at 512 threads, no spills), so a pass touches no shared memory
// outside its reduction: measured at 128^3 the pass fell from 3.53 to 3.31 us
// against z held in shared memory.  P pairs per thread; the rows of a block
// are its contiguous chunk (an even start, at most one unpaired last row).
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

template <int P, int BD>
__global__ void __launch_bounds__(BD, 1) k_mgs_res2(float* __restrict__ V, int64_t ldv, int n, GmresState* st,
                                                      double* H, double* cs, double* sn, double* g,
                                                      unsigned long long* tags, unsigned long long tmo, int giv,
                                                      int bulk) {
    constexpr bool kBulk = (int64_t)2 * P * BD * (int64_t)sizeof(float) >= kBulkPollBytes;
    __shared__ float s_w[32];
    __shared__ float s_tot;
    __shared__ unsigned s_seq;
    __shared__ int s_ok, s_j, s_done, s_kmax;
    __shared__ __align__(16) unsigned long long s_slots[kBulk ? 2 * kTagMaxBlocks + 2 : 2];  // warp 0's copies
    __shared__ __align__(8) uint64_t s_mbar;
    unsigned phase = 0;
    if (threadIdx.x == 0) {
        s_j = st->j;
        s_done = st->done;
        s_kmax = st->kmax;
        s_seq = *(volatile unsigned*)&st->bar.seq;
        if (kBulk) {
            mbar_init(&s_mbar, 1);
            mbar_init_fence();
        }
    }
    __syncthreads();
    if (s_done) return;
    const int j = s_j, kmax = s_kmax;
    const unsigned seq0 = s_seq;
    const int G = gridDim.x - giv;  // blocks that hold rows and publish partial sums
    if (giv && blockIdx.x == G) {
        givens_block<float>(j, kmax, H, cs, sn, g, st, tags, G, seq0, tmo);
        return;
    }
    int64_t r0, r1;
    block_rows(n, G, r0, r1);
    const int nb = r1 > r0 ? (int)(r1 - r0) : 0;
    const int tid = threadIdx.x;
    // pair q covers rows 2q, 2q + 1 of the chunk; the second may lie past nb
    auto ld2 = [&](const float* p, int q) -> float2 {
        if (2 * q + 1 < nb) return *reinterpret_cast<const float2*>(p + 2 * q);
        return make_float2(p[2 * q], 0.0f);
    };
    float* z = V + (int64_t)(j + 1) * ldv + r0;
    const float* v0 = V + r0;
    // z (this thread's rows of the new vector), v_{i-1} and v_i in registers
    float2 zr[P], vcur[P], vnext[P];
    const float2 zero2 = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int t = 0; t < P; ++t) {
        const int q = tid + t * BD;
        zr[t] = zero2;
        vcur[t] = zero2;
        vnext[t] = zero2;
        if (2 * q < nb) {
            zr[t] = ld2(z, q);
            vcur[t] = ld2(v0, q);
        }
    }
    float2 acc2 = zero2;
#pragma unroll
    for (int t = 0; t < P; ++t) {
        const int q = tid + t * BD;
        if (2 * q < nb) acc2 = __fadd2_rn(acc2, __fmul2_rn(vcur[t], zr[t]));
    }
    tag_arrive(__fadd_rn(acc2.x, acc2.y), tags, 0, seq0 + 1u, s_w, G);
    for (int i = 1; i <= j + 1; ++i) {
        if (i <= j) {
            const float* vi = V + (int64_t)i * ldv + r0;
#pragma unroll
            for (int t = 0; t < P; ++t) {
                const int q = tid + t * BD;
                if (2 * q < nb) vnext[t] = ld2(vi, q);
            }
        }
        const float h = tag_wait_bulk(tags, (i - 1) & 1, seq0 + (unsigned)i, &st->bar, tmo, &s_tot, &s_ok, G,
                                      s_slots, &s_mbar, phase, kBulk && bulk);
        if (!s_ok) {
            if (blockIdx.x == 0 && tid == 0) {
                st->status = BSPAI_TIMEOUT;
                st->done = 1;
            }
            return;
        }
        if (!giv && blockIdx.x == 0 && tid == 0) H[(int64_t)j * (kmax + 1) + (i - 1)] = (double)h;
        const float2 h2 = make_float2(h, h);
        acc2 = zero2;
#pragma unroll
        for (int t = 0; t < P; ++t) {
            const int q = tid + t * BD;
            if (2 * q < nb) {
                zr[t] = f2_sub(zr[t], __fmul2_rn(h2, vcur[t]));
                acc2 = __fadd2_rn(acc2, __fmul2_rn(i <= j ? vnext[t] : zr[t], zr[t]));
            }
        }
        tag_arrive(__fadd_rn(acc2.x, acc2.y), tags, i & 1, seq0 + (unsigned)i + 1u, s_w, G);
#pragma unroll
        for (int t = 0; t < P; ++t) vcur[t] = vnext[t];
    }
    const float hz = tag_wait_bulk(tags, (j + 1) & 1, seq0 + (unsigned)j + 2u, &st->bar, tmo, &s_tot, &s_ok, G,
                                   s_slots, &s_mbar, phase, kBulk && bulk);
    if (!s_ok) {
        if (blockIdx.x == 0 && tid == 0) {
            st->status = BSPAI_TIMEOUT;
            st->done = 1;
        }
        return;
    }
    // (with a Givens block, that block advances it: it may have started last)
    if (!giv && blockIdx.x == 0 && tid == 0) st->bar.seq = seq0 + (unsigned)j + 2u;
    const float hn = __fsqrt_rn(hz);
    const bool norm = hn > 0.0f && isfinite((double)hn);
#pragma unroll
    for (int t = 0; t < P; ++t) {
        const int q = tid + t * BD;
        if (2 * q < nb) {
            float2 zo = zr[t];
            if (norm) zo = make_float2(__fdiv_rn(zo.x, hn), __fdiv_rn(zo.y, hn));
            if (2 * q + 1 < nb) *reinterpret_cast<float2*>(z + 2 * q) = zo;
            else z[2 * q] = zo.x;
        }
    }
    if (!giv && blockIdx.x == 0 && tid == 0) givens_step(j, kmax, (double)hn, H, cs, sn, g, st);
}

// ---------------------------------------------------------------- host side
struct HostFlags {
    int j, done, status, kmax;
};

struct GmresWork;
static int choose_mgs(GmresWork& W);

struct GmresWork {
    int n = 0, kmax = 0, G = 0, ug = BSPAI_FP32, up = BSPAI_FP32;
    int64_t ldv = 0;
    void* V = nullptr;
    void* w = nullptr;
    void* part = nullptr;
    unsigned long long* tags = nullptr;  // k_mgs_res slots: 2 parities x blocks x 2 words
    GmresState* st = nullptr;
    double *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr, *norms = nullptr;
    HostFlags* hflags = nullptr;  // pinned
    unsigned long long tmo_ns = 2000000000ull;
    const bspai_bucketed* BA = nullptr;  // bucketed A for A v (null: A in u_p)
    int u32 = 0;                         // working precision u = fp32: d and x rounded to fp32
    void* res_fn = nullptr;  // k_mgs_res instance, or null for k_mgs
    int res_bd = 1024;       // its block size
    int res_kind = 0;        // 1: k_mgs_res, 2: k_mgs_res2 (see ResInstance)
    int res_per_thread = 0;  // its rows (k_mgs_res) or row pairs (k_mgs_res2) per thread
    int Gr = 0;              // its blocks that hold rows (at most one block per SM)
    int giv = 0;             // 1: one more block applies the Givens rotations during the passes
    int bulk = 0;            // 1: an instance able to poll by bulk copies does (see kBulkPollBytes)
    size_t res_smem = 0;
    cudaStream_t s = nullptr;

    static size_t tag_words() { return (size_t)4 * kTagMaxBlocks; }
    int sms = 0;  // SMs the cooperative kernels may use (one block of k_mgs_res each)
    int alloc(int n_, int kmax_, int ug_, int up_, double timeout_s, int max_blocks, cudaStream_t st_) {
        sms = max_blocks > 0 && max_blocks < num_sms() ? max_blocks : num_sms();
        n = n_;
        kmax = kmax_;
        ug = ug_;
        up = up_;
        s = st_;
        tmo_ns = (unsigned long long)((timeout_s > 0 ? timeout_s : 2.0) * 1e9);
        const size_t es = ug == BSPAI_FP64 ? 8 : 4;
        ldv = ceil_div(n > 0 ? n : 1, 64) * 64;
        int occ = 0;
        cudaError_t e;
        if (ug == BSPAI_FP64) {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mgs<double>, 512, 0);
            int occ2 = 0;
            if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_gmres_start<double>, 512, 0);
            occ = occ < occ2 ? occ : occ2;
        } else {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mgs<float>, 512, 0);
            int occ2 = 0;
            if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_gmres_start<float>, 512, 0);
            occ = occ < occ2 ? occ : occ2;
        }
        if (e) return cuda_error(e, "occupancy", __FILE__, __LINE__);
        if (occ < 1) return set_error(BSPAI_ERR_CUDA, "gmres: cooperative kernel does not fit on an SM");
        G = (occ >= 2 ? 2 : 1) * sms;
        BSPAI_TRY(dalloc(&V, es * (size_t)ldv * (size_t)(kmax + 1), s));
        BSPAI_TRY(dalloc(&w, es * (size_t)ldv, s));
        BSPAI_TRY(dalloc(&part, es * 2 * (size_t)G, s));
        BSPAI_TRY(dalloc_t(&tags, tag_words(), s));
        CUDA_TRY(cudaMemsetAsync(tags, 0, sizeof(unsigned long long) * tag_words(), s));
        BSPAI_TRY(dalloc_t(&st, 1, s));
        BSPAI_TRY(dalloc_t(&H, (size_t)(kmax + 1) * kmax, s));
        BSPAI_TRY(dalloc_t(&cs, (size_t)kmax + 1, s));
        BSPAI_TRY(dalloc_t(&sn, (size_t)kmax + 1, s));
        BSPAI_TRY(dalloc_t(&g, (size_t)kmax + 2, s));
        BSPAI_TRY(dalloc_t(&y, (size_t)kmax + 1, s));
        BSPAI_TRY(dalloc_t(&norms, 4, s));
        CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(GmresState), s));
        CUDA_TRY(cudaMemsetAsync(g, 0, sizeof(double) * ((size_t)kmax + 2), s));
        // one pinned flag word per host thread, kept for the life of the process
        static thread_local HostFlags* t_flags = nullptr;
        if (!t_flags) CUDA_TRY(cudaMallocHost(&t_flags, sizeof(HostFlags)));
        hflags = t_flags;
        return choose_mgs(*this);
    }
    void release() {
        dfree(V, s); dfree(w, s); dfree(part, s); dfree(tags, s); dfree(st, s); dfree(H, s); dfree(cs, s);
        dfree(sn, s); dfree(g, s); dfree(y, s); dfree(norms, s);
        V = w = part = nullptr;
        tags = nullptr;
        st = nullptr;
        H = cs = sn = g = y = norms = nullptr;
    }
};

// One k_mgs_res / k_mgs_res2 instance: its kernel, kind (1: k_mgs_res, rows of a
// thread one by one; 2: k_mgs_res2, rows in packed pairs), rows (R) or pairs (P)
// per thread, and block size.  The instance is the smallest that holds a
// block's chunk of rows: every instance listed here is reachable from
// choose_mgs for some order n (the parity tests run each one).
struct ResInstance {
    void* fn = nullptr;
    int kind = 0, per_thread = 0, bd = 0;
};

template <typename T>
static ResInstance pick_res(int64_t chunk) {
    const int R = (int)ceil_div(chunk, 1024);
    if (R <= 1) return {(void*)k_mgs_res<T, 1, 1024>, 1, 1, 1024};
    if constexpr (sizeof(T) == 4) {
        // fp32: rows in adjacent pairs, packed two-lane arithmetic
        if (R <= 2) return {(void*)k_mgs_res2<1, 1024>, 2, 1, 1024};
        if (R <= 4) return {(void*)k_mgs_res2<2, 1024>, 2, 2, 1024};
        if (R <= 8) return {(void*)k_mgs_res2<4, 1024>, 2, 4, 1024};
        // more rows per block: 512 threads with more pairs each (chunk > 8192)
        const int Rp = (int)ceil_div(chunk, 512);
        if (Rp <= 24) return {(void*)k_mgs_res2<12, 512>, 2, 12, 512};
        if (Rp <= 28) return {(void*)k_mgs_res2<14, 512>, 2, 14, 512};
        if (Rp <= 32) return {(void*)k_mgs_res2<16, 512>, 2, 16, 512};
        return {};
    } else {
        // fp64: z in shared memory, at most 8192 rows of a block (64 KB)
        if (R <= 2) return {(void*)k_mgs_res<T, 2, 1024>, 1, 2, 1024};
        if (R <= 4) return {(void*)k_mgs_res<T, 4, 1024>, 1, 4, 1024};
        if (R <= 8) return {(void*)k_mgs_res<T, 8, 1024>, 1, 8, 1024};
        return {};
    }
}

// Use the on-chip MGS kernel when one block per SM can hold its rows of z on
// chip (fp32: in registers; fp64: in shared memory, at most 200 KB) with at
// most 32 (fp32) / 16 (fp64) rows per thread of a 512-thread block.
static int choose_mgs(GmresWork& W) {
    W.res_fn = nullptr;
    // As few blocks as hold the rows of z on chip, but not fewer than kMgsBlocks: each
    // grid reduction of the j + 2 per Arnoldi step waits for every block, and fewer
    // blocks shorten it (measured per pass, n = 65,536 / 262,144: 2.5 / 3.1 us at 152
    // blocks, 1.6 / 1.9 us at 64) while one block still streams its rows faster than
    // the reduction completes.
    // rows per block of the largest instance.  At 128^3 fewer blocks stopped paying: 103
    // blocks of 40 fp32 rows per thread solved in 90.8 ms against 87.7 ms at 128 blocks of
    // 32 (the longer per-block update outweighs the shorter reduction), and a scalar
    // 768-thread instance (22,272 rows, register spills) took 107.6 ms at 95 blocks.
    const int64_t cap = W.ug == BSPAI_FP64 ? 8192 : 16384;
    int Gr = (int)ceil_div(W.n, cap);
    if (Gr < kMgsBlocks) Gr = kMgsBlocks;
    if (Gr > W.sms) Gr = W.sms;
    if (Gr > kTagMaxBlocks) return BSPAI_OK;
    const int64_t chunk = ceil_div(ceil_div(W.n, Gr), 32) * 32;
    const size_t es = W.ug == BSPAI_FP64 ? 8 : 4;
    const size_t smem = (size_t)chunk * es;
    if (smem > 200 * 1024) return BSPAI_OK;
    const ResInstance ri = es == 8 ? pick_res<double>(chunk) : pick_res<float>(chunk);
    if (!ri.fn) return BSPAI_OK;
    CUDA_TRY(cudaFuncSetAttribute(ri.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ri.fn, ri.bd, smem));
    if (occ < 1) return BSPAI_OK;
    W.res_fn = ri.fn;
    W.res_bd = ri.bd;
    W.res_kind = ri.kind;
    W.res_per_thread = ri.per_thread;
    W.Gr = Gr;
    // the Givens block needs an SM of its own (one block per SM at these sizes)
    W.giv = Gr + 1 <= W.sms ? 1 : 0;
    // bulk-copy polling where it was measured to pay: at least kMgsBlocks blocks (a solve
    // confined to a few SMs, as each of several concurrent right-hand sides is, polls few
    // slots and the copy engine's round trip loses) and kBulkPollBytes of a vector per block
    W.bulk = Gr >= kMgsBlocks && (int64_t)chunk * (int64_t)es >= kBulkPollBytes ? 1 : 0;
    W.res_smem = smem;
    return BSPAI_OK;
}

static int coop_launch_cfg(void* fn, int G, int block, size_t smem, void** args, cudaStream_t s) {
    cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(G), dim3(block), args, smem, s);
    note_launch();
    if (e) return cuda_error(e, "cudaLaunchCooperativeKernel", __FILE__, __LINE__);
    return BSPAI_OK;
}

static int coop_launch(void* fn, int G, void** args, cudaStream_t s) {
    cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(G), dim3(512), args, 0, s);
    note_launch();
    if (e) return cuda_error(e, "cudaLaunchCooperativeKernel", __FILE__, __LINE__);
    return BSPAI_OK;
}

struct GmresResult {
    int k = 0;
    int status = BSPAI_OK;
    double beta = 0.0, res = 0.0, dmax = 0.0, xmax = 0.0;
};

// One GMRES solve of (M A) d = M r.  x != null: x += d; dout != null: d out.
template <typename T>
static int gmres_run(GmresWork& W, const bspai_matrix* A, const bspai_bucketed* BM, const double* r, double tau,
                     double* x, double* dout, GmresResult& out, double target = 0.0) {
    cudaStream_t s = W.s;
    const int n = W.n;
    const int tprec = W.ug;  // T matches u_g
    // A v: A in u_p, or A's buckets by the adaptive-precision SpMV (Alg 2.3 applied to A)
    const BMDev Aview = W.BA ? W.BA->dev() : up_view(A, W.up);
    const BMDev Mview = BM->dev();
    T* V = reinterpret_cast<T*>(W.V);
    T* w = reinterpret_cast<T*>(W.w);
    T* part = reinterpret_cast<T*>(W.part);
    {
        ProfScope ps(BSPAI_K_OTHER, s);
        k_state_init<<<1, 1, 0, s>>>(W.st, W.kmax, tau, target);
        note_launch();
        CUDA_LAUNCH_CHECK();
        CUDA_TRY(cudaMemsetAsync(W.norms, 0, 4 * sizeof(double), s));
    }
    {
        ProfScope ps(BSPAI_K_BSPMV, s);
        BSPAI_TRY(launch_bspmv(Mview, r, BSPAI_FP64, V, tprec, s));
    }
    {
        ProfScope ps(BSPAI_K_MGS, s);
        int nn = n;
        void* args[] = {&V, &nn, &W.st, &W.g, &part, &W.tmo_ns};
        BSPAI_TRY(coop_launch((void*)k_gmres_start<T>, W.G, args, s));
    }
    int launched = 0, chunk = 4;
    const int* jd = &W.st->j;
    while (launched < W.kmax) {
        for (int c = 0; c < chunk && launched < W.kmax; ++c, ++launched) {
            {
                ProfScope ps(BSPAI_K_SPMV_A, s);
                BSPAI_TRY(launch_bspmv_idx(Aview, V, tprec, w, tprec, jd, W.ldv, 0, 0, s));
            }
            {
                ProfScope ps(BSPAI_K_BSPMV, s);
                BSPAI_TRY(launch_bspmv_idx(Mview, w, tprec, V, tprec, jd, 0, W.ldv, 1, s));
            }
            {
                ProfScope ps(BSPAI_K_MGS, s);
                int nn = n;
                int64_t ld = W.ldv;
                if (W.res_fn) {
                    void* args[] = {&V, &ld, &nn, &W.st, &W.H, &W.cs, &W.sn, &W.g, &W.tags, &W.tmo_ns, &W.giv,
                                    &W.bulk};
                    BSPAI_TRY(coop_launch_cfg(W.res_fn, W.Gr + W.giv, W.res_bd, W.res_smem, args, s));
                } else {
                    void* args[] = {&V, &ld, &nn, &W.st, &W.H, &W.cs, &W.sn, &W.g, &part, &W.tmo_ns};
                    BSPAI_TRY(coop_launch((void*)k_mgs<T>, W.G, args, s));
                }
            }
        }
        CUDA_TRY(cudaMemcpyAsync(W.hflags, W.st, sizeof(HostFlags), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        if (W.hflags->done) break;
        chunk = chunk < 32 ? chunk * 2 : 32;
    }
    {
        ProfScope ps(BSPAI_K_UPDATE, s);
        k_backsolve<<<1, kBackThreads, kBackSmem, s>>>(W.st, W.H, W.g, W.y, W.kmax);
        note_launch();
        CUDA_LAUNCH_CHECK();
        if (n > 0) {
            k_gmres_update<T><<<wave_grid(n), 256, sizeof(T) * (size_t)(W.kmax + 1), s>>>(
                V, W.ldv, n, W.st, W.y, x, dout, W.norms, W.u32);
            note_launch();
            CUDA_LAUNCH_CHECK();
        }
    }
    GmresState hs;
    double hn[2];
    CUDA_TRY(cudaMemcpyAsync(&hs, W.st, sizeof hs, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(hn, W.norms, sizeof hn, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    BSPAI_TRY(stage_timeout_take(s));
    out.k = hs.j;
    out.status = hs.status;
    out.beta = hs.beta;
    out.res = hs.res;
    out.dmax = hn[0];
    out.xmax = hn[1];
    if (hs.status == BSPAI_TIMEOUT) {
        // the barrier state is undefined after a timeout: reset it (and the
        // tagged slots, whose numbers restart with it) for reuse
        CUDA_TRY(cudaMemsetAsync(&W.st->bar, 0, sizeof(GridBar), s));
        CUDA_TRY(cudaMemsetAsync(W.tags, 0, sizeof(unsigned long long) * GmresWork::tag_words(), s));
        return set_error(BSPAI_TIMEOUT, "gmres: a grid barrier exceeded its time limit");
    }
    return BSPAI_OK;
}

static int check_solver_precs(int u, int u_r, int u_g, int u_p) {
    if (u != BSPAI_FP64 && u != BSPAI_FP32)
        return set_error(BSPAI_ERR_UNSUPPORTED, "working precision u must be FP64 or FP32");
    if (u_r != BSPAI_DD && u_r != BSPAI_FP64) return set_error(BSPAI_ERR_UNSUPPORTED, "u_r must be DD or FP64");
    if (u_g != BSPAI_FP32 && u_g != BSPAI_FP64) return set_error(BSPAI_ERR_UNSUPPORTED, "u_g must be FP32 or FP64");
    if (u_p != BSPAI_FP32 && u_p != BSPAI_FP64) return set_error(BSPAI_ERR_UNSUPPORTED, "u_p must be FP32 or FP64");
    return BSPAI_OK;
}

static constexpr int kKmaxLimit = 4000;  // shared-memory bound of k_backsolve / k_gmres_update

static int resolve_kmax(const bspai_opts_t* o, int n) {
    int k = o && o->kmax > 0 ? o->kmax : (n < 1000 ? n : 1000);
    if (k > n) k = n;
    if (k > kKmaxLimit) k = kKmaxLimit;
    return k < 1 ? 1 : k;
}

int launch_residual_prec(const bspai_matrix* A, const double* x, const double* b, double* r, double* norms,
                         int u_r, int u, cudaStream_t s);

__global__ void k_round_f32(int n, double* __restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = (double)__double2float_rn(x[i]);
}

// d += e in fp64 (e, a restarted cycle's correction, already stored in u); first: d = 0 + e
__global__ void k_dacc_add(int n, double* __restrict__ d, const double* __restrict__ e, int first) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = __dadd_rn(first ? 0.0 : d[i], e[i]);
}

// x = fl_u(x + fl_u(d)) for a correction summed over restarted cycles, with
// norms[0] = max |fl_u(d)|, norms[1] = max |x| (as k_gmres_update)
__global__ void __launch_bounds__(256) k_apply_d(int n, double* __restrict__ x, const double* __restrict__ d,
                                                 double* __restrict__ norms, int u32) {
    double dabs = 0.0, xabs = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double dv = d[r];
        if (u32) dv = (double)__double2float_rn(dv);
        double xn = __dadd_rn(x[r], dv);
        if (u32) xn = (double)__double2float_rn(xn);
        x[r] = xn;
        double da = fabs(dv), xa = fabs(xn);
        if (!(da <= 1.7976931348623157e308)) da = __longlong_as_double(0x7ff0000000000000LL);
        if (!(xa <= 1.7976931348623157e308)) xa = __longlong_as_double(0x7ff0000000000000LL);
        dabs = fmax(dabs, da);
        xabs = fmax(xabs, xa);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dabs = fmax(dabs, __shfl_xor_sync(0xffffffffu, dabs, o));
        xabs = fmax(xabs, __shfl_xor_sync(0xffffffffu, xabs, o));
    }
    block_atomic_max_nonneg2(norms, dabs, norms + 1, xabs);
}

static int ir_solve(bspai_matrix* A, const bspai_bucketed* BA, const double* b, const bspai_bucketed* BM,
                    const bspai_spai* M, int u, int u_r, int u_g, int u_p, double tol, const bspai_opts_t* opts,
                    double* x, cudaStream_t s, bspai_solve_info_t* info) {
    bspai_opts_t o;
    bspai_opts_default(&o);
    if (opts) o = *opts;
    const int n = A->n;
    const int kmax = resolve_kmax(&o, n);
    int imax = o.i_max > 0 ? o.i_max : 10;
    if (imax > 32) imax = 32;
    const double ustop = o.u_stop > 0 ? o.u_stop : (u == BSPAI_FP32 ? 0x1p-24 : 0x1p-53);
    const double stag = o.stagnation > 0 ? o.stagnation : 0.9;
    const double tau = tol > 0 ? tol : o.tau;
    bspai_solve_info_t inf;
    memset(&inf, 0, sizeof inf);
    if (BM->n != n || (M && M->n != n)) return set_error(BSPAI_ERR_INVALID, "gmres_ir_solve: size mismatch");
    if (!o.x0_given && !M) return set_error(BSPAI_ERR_INVALID, "gmres_ir_solve: need M for x0 = M b");
    if (n == 0) {
        if (info) *info = inf;
        return BSPAI_OK;
    }
    double* r = nullptr;
    double* nrm = nullptr;
    double *dacc = nullptr, *ecyc = nullptr, *rcyc = nullptr;  // restarted cycles only
    GmresWork W;
    int rc = BSPAI_OK;
    auto finish = [&](int code) {
        dfree(r, s);
        dfree(nrm, s);
        dfree(dacc, s);
        dfree(ecyc, s);
        dfree(rcyc, s);
        W.release();
        inf.status = code;
        if (info) *info = inf;
        return code;
    };
    // the Krylov basis: kmax + 1 vectors, or fewer (restarted cycles) when the caller's
    // byte cap or the device's free memory asks
    int km = kmax;
    if (o.basis_bytes_max > 0) {
        const int64_t vec = (int64_t)(u_g == BSPAI_FP64 ? 8 : 4) * (ceil_div(n, 64) * 64);
        const int64_t fit = o.basis_bytes_max / vec - 1;
        if (fit < 1)
            return finish(set_error(BSPAI_ERR_INVALID,
                                    "gmres_ir_solve: basis_bytes_max holds fewer than two Krylov vectors of order %d",
                                    n));
        if (fit < km) km = (int)fit;
    }
    if ((rc = dalloc_t(&r, (size_t)n, s))) return finish(rc);
    if ((rc = dalloc_t(&nrm, 4, s))) return finish(rc);
    rc = W.alloc(n, km, u_g, u_p, o.barrier_timeout_s, o.max_blocks, s);
    while (rc == BSPAI_ERR_NOMEM && km > 8) {
        W.release();
        (void)cudaGetLastError();  // the failed allocation's error is not the next launch's
        km = km / 2 > 8 ? km / 2 : 8;
        rc = W.alloc(n, km, u_g, u_p, o.barrier_timeout_s, o.max_blocks, s);
    }
    if (rc) return finish(rc);
    if (km < kmax) {
        if ((rc = dalloc_t(&dacc, (size_t)n, s))) return finish(rc);
        if ((rc = dalloc_t(&ecyc, (size_t)n, s))) return finish(rc);
        if ((rc = dalloc_t(&rcyc, (size_t)n, s))) return finish(rc);
    }
    inf.kmem = km;
    W.BA = BA;
    W.u32 = u == BSPAI_FP32;
    // ||A||_inf, ||b||_inf
    double anorm = 0.0, bnorm = 0.0;
    {
        ProfScope ps(BSPAI_K_OTHER, s);
        cudaError_t e0 = cudaMemsetAsync(nrm, 0, 4 * sizeof(double), s);
        if (e0) return finish(cuda_error(e0, "memset", __FILE__, __LINE__));
        k_absmax<<<wave_grid(n), 256, 0, s>>>(n, b, nrm);
        note_launch();
        if (!o.x0_given) {
            // x0 = M b with the unbucketed M in u_f (fp32 or fp16), stored in fp64
            if ((rc = launch_apply_uf(M, b, x, s))) return finish(rc);
        } else if (W.u32) {
            // a given x0 is held in u = fp32 (M b in u_f <= fp32 already is)
            k_round_f32<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, x);
            note_launch();
        }
    }
    cudaError_t e = cudaMemcpyAsync(&bnorm, nrm, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(&anorm, A->norm_inf, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return finish(cuda_error(e, "norms", __FILE__, __LINE__));
    double dprev = INFINITY;
    int code = BSPAI_NOT_CONVERGED;
    for (int i = 0; i < imax; ++i) {
        double hn[2] = {0, 0};
        e = cudaMemsetAsync(nrm, 0, 2 * sizeof(double), s);
        if (e) return finish(cuda_error(e, "memset", __FILE__, __LINE__));
        if ((rc = launch_residual_prec(A, x, b, r, nrm, u_r, u, s))) return finish(rc);
        e = cudaMemcpyAsync(hn, nrm, sizeof hn, cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) return finish(cuda_error(e, "residual norms", __FILE__, __LINE__));
        // a zero residual is an exact solution (b = 0, x = 0 gives 0 / 0 otherwise)
        const double nbe = hn[0] == 0.0 ? 0.0 : hn[0] / (anorm * hn[1] + bnorm);
        inf.nbe[i] = nbe;
        if (!std::isfinite(nbe)) {
            code = set_error(BSPAI_NONFINITE, "gmres_ir_solve: non-finite residual at step %d", i);
            break;
        }
        if (nbe <= ustop) {
            inf.stop_reason = 1;
            code = BSPAI_OK;
            break;
        }
        GmresResult gr;
        int cycles = 1;
        if (km >= kmax) {
            rc = u_g == BSPAI_FP64 ? gmres_run<double>(W, A, BM, r, tau, x, nullptr, gr)
                                   : gmres_run<float>(W, A, BM, r, tau, x, nullptr, gr);
            if (rc) return finish(rc);
        } else {
            // restarted cycles of km steps on the correction equation A d = r: cycle c > 0
            // starts from r - A d (u_r, stored in u) and stops at cycle 0's level tau beta_0
            int steps = 0;
            double lvl = 0.0, beta0 = 0.0;
            GmresResult gc;
            cycles = 0;
            while (steps < kmax) {
                const double* rin = r;
                if (cycles > 0) {
                    e = cudaMemsetAsync(nrm + 2, 0, 2 * sizeof(double), s);
                    if (e) return finish(cuda_error(e, "memset", __FILE__, __LINE__));
                    if ((rc = launch_residual_prec(A, dacc, r, rcyc, nrm + 2, u_r, u, s))) return finish(rc);
                    rin = rcyc;
                }
                rc = u_g == BSPAI_FP64 ? gmres_run<double>(W, A, BM, rin, tau, nullptr, ecyc, gc, lvl)
                                       : gmres_run<float>(W, A, BM, rin, tau, nullptr, ecyc, gc, lvl);
                if (rc) return finish(rc);
                if (cycles == 0) {
                    beta0 = gc.beta;
                    lvl = tau * beta0;
                }
                k_dacc_add<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, dacc, ecyc, cycles == 0);
                note_launch();
                steps += gc.k;
                ++cycles;
                if (gc.status == BSPAI_NONFINITE || gc.k < km || gc.res <= lvl || !(gc.beta > 0.0)) break;
            }
            {
                ProfScope ps(BSPAI_K_UPDATE, s);
                e = cudaMemsetAsync(W.norms, 0, 2 * sizeof(double), s);
                if (e) return finish(cuda_error(e, "memset", __FILE__, __LINE__));
                k_apply_d<<<wave_grid(n), 256, 0, s>>>(n, x, dacc, W.norms, W.u32);
                note_launch();
            }
            double hn2[2];
            e = cudaMemcpyAsync(hn2, W.norms, sizeof hn2, cudaMemcpyDeviceToHost, s);
            if (!e) e = cudaStreamSynchronize(s);
            if (e) return finish(cuda_error(e, "restarted GMRES update", __FILE__, __LINE__));
            gr.k = steps;
            gr.status = gc.status;
            gr.beta = beta0;
            gr.res = gc.res;
            gr.dmax = hn2[0];
            gr.xmax = hn2[1];
        }
        inf.gmres_cycles[i] = cycles;
        inf.gmres_iters[i] = gr.k;
        inf.total_iters += gr.k;
        inf.relres[i] = gr.beta > 0 ? gr.res / gr.beta : 0.0;
        inf.ir_steps = i + 1;
        inf.dx[i] = gr.xmax > 0 ? gr.dmax / gr.xmax : gr.dmax;
        if (gr.status == BSPAI_NONFINITE || !std::isfinite(gr.dmax) || !std::isfinite(gr.xmax)) {
            code = set_error(BSPAI_NONFINITE, "gmres_ir_solve: non-finite value in GMRES at step %d", i);
            break;
        }
        if (gr.dmax <= ustop * gr.xmax) {
            inf.stop_reason = 2;
            code = BSPAI_OK;
            break;
        }
        if (i > 0 && gr.dmax > stag * dprev) {
            inf.stop_reason = 3;
            code = BSPAI_OK;
            break;
        }
        dprev = gr.dmax;
    }
    if (code == BSPAI_NOT_CONVERGED) set_error(code, "gmres_ir_solve: i_max = %d steps without meeting a stopping test", imax);
    return finish(code);
}

// Failure-detection self-test: the bounded grid barrier, its arrival counter
// pre-loaded past the value at which the last arrival releases it (hold != 0),
// so that no arrival releases it and every block's wait must run out.
__global__ void k_barrier_selftest(GridBar* bar, unsigned long long tmo, int* failed) {
    const bool ok = grid_sync(bar, tmo);
    if (!ok && threadIdx.x == 0) atomicExch(failed, 1);
}

}  // namespace bspai

using namespace bspai;

extern "C" {

int bspai_barrier_selftest(int blocks, int hold, double timeout_s, bspai_stream_t st, float* waited_ms) {
    cudaStream_t s = (cudaStream_t)st;
    if (blocks < 1 || blocks > 1024 || !(timeout_s > 0) || timeout_s > 10)
        return set_error(BSPAI_ERR_INVALID, "barrier self-test: bad arguments");
    int dev = 0, coop = 0, per_sm = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_barrier_selftest, 32, 0));
    if (!coop || blocks > per_sm * num_sms())
        return set_error(BSPAI_ERR_INVALID, "barrier self-test: blocks cannot be co-resident");
    void* p = nullptr;
    int rc = dalloc(&p, sizeof(GridBar) + sizeof(int), s);
    if (rc) return rc;
    GridBar* bar = (GridBar*)p;
    int* failed = (int*)(bar + 1);
    GridBar init{hold ? (unsigned)blocks : 0u, 0u, 0, 0};  // arrivals count from here
    int h_failed = 0;
    float ms = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMemcpyAsync(bar, &init, sizeof init, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemsetAsync(failed, 0, sizeof(int), s);
    if (!e) e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    if (!e) e = cudaEventRecord(e0, s);
    if (!e) {
        unsigned long long tmo = (unsigned long long)(timeout_s * 1e9);
        void* args[] = {&bar, &tmo, &failed};
        e = cudaLaunchCooperativeKernel((const void*)k_barrier_selftest, dim3(blocks), dim3(32), args, 0, s);
        note_launch();
    }
    if (!e) e = cudaEventRecord(e1, s);
    if (!e) e = cudaMemcpyAsync(&h_failed, failed, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dfree(p, s);
    if (e) return cuda_error(e, "barrier self-test", __FILE__, __LINE__);
    if (waited_ms) *waited_ms = ms;
    if (h_failed) return set_error(BSPAI_TIMEOUT, "barrier self-test: the grid barrier timed out");
    return BSPAI_OK;
}

int gmres_ir_solve_h(bspai_A_h A, const double* b, bspai_BM_h BM, bspai_M_h M, bspai_prec_t u, bspai_prec_t u_r,
                     bspai_prec_t u_g, bspai_prec_t u_p, double tol, const bspai_opts_t* opts, double* x,
                     bspai_stream_t s, bspai_solve_info_t* info) {
    if (!A || A->magic != kMagicA) return set_error(BSPAI_ERR_INVALID, "gmres_ir_solve: bad A handle");
    if (!BM || BM->magic != kMagicBM) return set_error(BSPAI_ERR_INVALID, "gmres_ir_solve: bad bucketed M handle");
    if (M && M->magic != kMagicM) return set_error(BSPAI_ERR_INVALID, "gmres_ir_solve: bad M handle");
    if (A->n > 0 && (!b || !x)) return set_error(BSPAI_ERR_INVALID, "gmres_ir_solve: null vector");
    BSPAI_TRY(check_solver_precs(u, u_r, u_g, u_p));
    return ir_solve(A, nullptr, b, BM, M, u, u_r, u_g, u_p, tol, opts, x, (cudaStream_t)s, info);
}

int gmres_ir_solve_hb(bspai_A_h A, bspai_BM_h A_bucketed, const double* b, bspai_BM_h BM, bspai_M_h M,
                      bspai_prec_t u, bspai_prec_t u_r, bspai_prec_t u_g, double tol, const bspai_opts_t* opts,
                      double* x, bspai_stream_t s, bspai_solve_info_t* info) {
    if (!A || A->magic != kMagicA) return set_error(BSPAI_ERR_INVALID, "gmres_ir_solve_hb: bad A handle");
    if (!A_bucketed || A_bucketed->magic != kMagicBM || A_bucketed->n != A->n)
        return set_error(BSPAI_ERR_INVALID, "gmres_ir_solve_hb: bad bucketed A handle");
    if (!BM || BM->magic != kMagicBM) return set_error(BSPAI_ERR_INVALID, "gmres_ir_solve_hb: bad bucketed M handle");
    if (M && M->magic != kMagicM) return set_error(BSPAI_ERR_INVALID, "gmres_ir_solve_hb: bad M handle");
    if (A->n > 0 && (!b || !x)) return set_error(BSPAI_ERR_INVALID, "gmres_ir_solve_hb: null vector");
    BSPAI_TRY(check_solver_precs(u, u_r, u_g, u_g));
    return ir_solve(A, A_bucketed, b, BM, M, u, u_r, u_g, u_g, tol, opts, x, (cudaStream_t)s, info);
}

int gmres_ir_solve(const bspai_csr_t* Acsr, const double* b, bspai_BM_h BM, bspai_M_h M, bspai_prec_t u,
                   bspai_prec_t u_r, bspai_prec_t u_g, bspai_prec_t u_p, double tol, const bspai_opts_t* opts,
                   double* x, bspai_stream_t s, bspai_solve_info_t* info) {
    BSPAI_TRY(check_solver_precs(u, u_r, u_g, u_p));
    bspai_matrix* A = nullptr;
    BSPAI_TRY(matrix_create(Acsr, (cudaStream_t)s, &A));
    int rc = gmres_ir_solve_h(A, b, BM, M, u, u_r, u_g, u_p, tol, opts, x, s, info);
    bspai_free(A);
    return rc;
}

static int gmres_one(bspai_matrix* A, const bspai_bucketed* BA, const bspai_bucketed* BM, const double* r,
                     bspai_prec_t u_g, bspai_prec_t u_p, const bspai_opts_t* opts, double* d, bspai_stream_t st,
                     bspai_solve_info_t* info) {
    cudaStream_t s = (cudaStream_t)st;
    if (!A || A->magic != kMagicA) return set_error(BSPAI_ERR_INVALID, "bspai_gmres: bad A handle");
    if (!BM || BM->magic != kMagicBM) return set_error(BSPAI_ERR_INVALID, "bspai_gmres: bad M handle");
    if (BM->n != A->n) return set_error(BSPAI_ERR_INVALID, "bspai_gmres: size mismatch");
    if (A->n > 0 && (!r || !d)) return set_error(BSPAI_ERR_INVALID, "bspai_gmres: null vector");
    BSPAI_TRY(check_solver_precs(BSPAI_FP64, BSPAI_DD, u_g, u_p));
    bspai_opts_t o;
    bspai_opts_default(&o);
    if (opts) o = *opts;
    bspai_solve_info_t inf;
    memset(&inf, 0, sizeof inf);
    if (A->n == 0) {
        if (info) *info = inf;
        return BSPAI_OK;
    }
    GmresWork W;
    int rc = W.alloc(A->n, resolve_kmax(&o, A->n), u_g, u_p, o.barrier_timeout_s, o.max_blocks, s);
    W.BA = BA;
    GmresResult gr;
    if (!rc)
        rc = u_g == BSPAI_FP64 ? gmres_run<double>(W, A, BM, r, o.tau, nullptr, d, gr)
                               : gmres_run<float>(W, A, BM, r, o.tau, nullptr, d, gr);
    W.release();
    inf.status = rc ? rc : gr.status;
    inf.ir_steps = 1;
    inf.gmres_iters[0] = gr.k;
    inf.total_iters = gr.k;
    inf.relres[0] = gr.beta > 0 ? gr.res / gr.beta : 0.0;
    if (info) *info = inf;
    if (!rc && gr.status == BSPAI_NONFINITE) return set_error(BSPAI_NONFINITE, "bspai_gmres: non-finite value");
    return rc;
}

int bspai_gmres_plan(int32_t n, bspai_prec_t u_g, int32_t max_blocks, bspai_gmres_plan_t* out) {
    if (!out) return set_error(BSPAI_ERR_INVALID, "bspai_gmres_plan: null out");
    memset(out, 0, sizeof *out);
    if (n < 1) return set_error(BSPAI_ERR_INVALID, "bspai_gmres_plan: n = %d", n);
    if (u_g != BSPAI_FP32 && u_g != BSPAI_FP64) return set_error(BSPAI_ERR_UNSUPPORTED, "u_g must be FP32 or FP64");
    GmresWork W;
    W.n = n;
    W.ug = u_g;
    W.sms = max_blocks > 0 && max_blocks < num_sms() ? max_blocks : num_sms();
    BSPAI_TRY(choose_mgs(W));
    if (W.res_fn) {
        out->kernel = W.res_kind;
        out->per_thread = W.res_per_thread;
        out->block_threads = W.res_bd;
        out->blocks = W.Gr;
        out->poll_bulk = W.bulk;
        return BSPAI_OK;
    }
    int occ = 0, occ2 = 0;
    cudaError_t e = u_g == BSPAI_FP64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mgs<double>, 512, 0)
                                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mgs<float>, 512, 0);
    if (!e)
        e = u_g == BSPAI_FP64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_gmres_start<double>, 512, 0)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_gmres_start<float>, 512, 0);
    if (e) return cuda_error(e, "occupancy", __FILE__, __LINE__);
    occ = occ < occ2 ? occ : occ2;
    out->kernel = 0;
    out->per_thread = 0;
    out->block_threads = 512;
    out->blocks = (occ >= 2 ? 2 : 1) * W.sms;
    return BSPAI_OK;
}

int bspai_gmres(bspai_A_h A, bspai_BM_h BM, const double* r, bspai_prec_t u_g, bspai_prec_t u_p,
                const bspai_opts_t* opts, double* d, bspai_stream_t st, bspai_solve_info_t* info) {
    return gmres_one(A, nullptr, BM, r, u_g, u_p, opts, d, st, info);
}

int bspai_gmres_b(bspai_A_h A, bspai_BM_h A_bucketed, bspai_BM_h BM, const double* r, bspai_prec_t u_g,
                  const bspai_opts_t* opts, double* d, bspai_stream_t st, bspai_solve_info_t* info) {
    if (!A_bucketed || A_bucketed->magic != kMagicBM || (A && A_bucketed->n != A->n))
        return set_error(BSPAI_ERR_INVALID, "bspai_gmres_b: bad bucketed A handle");
    return gmres_one(A, A_bucketed, BM, r, u_g, u_g, opts, d, st, info);
}

}  // extern "C"

// ---------------------------------------------------------------- no-allocation GMRES
// bspai_gmres_noalloc runs exactly the kernels of bspai_gmres, but takes its
// whole workspace (Krylov basis, Hessenberg matrix, rotations, partial sums,
// solver state) from one fixed block of device memory that is part of the
// library image, so it never asks the CUDA runtime for memory.  That block is
// set aside on every GPU that loads the library and stays there until the
// process exits.
namespace bspai {

constexpr size_t kNoallocScratchBytes = 64ull << 20;  // 64 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

static std::mutex g_noalloc_mu;
// Device address of the scratch per device ordinal, with the id of the CUDA
// context it was looked up in: after a device reset the module is loaded again
// in a new context (possibly at another address), so a cached address is used
// only while the current context is the one it came from.
struct NoallocAddr {
    unsigned long long ctx_id = 0;
    void* base = nullptr;
};
static NoallocAddr g_noalloc_base[128];

// The current context's process-unique id through the driver entry points
// (the library links the CUDA runtime only); false if they are unavailable.
static bool current_context_id(unsigned long long* id) {
    typedef int (*GetCurrentFn)(void**);
    typedef int (*GetIdFn)(void*, unsigned long long*);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetIdFn>(f);
    });
    void* ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, id) == 0;
}

// The host-side name of a __device__ array is only a stand-in, not a device
// address: the address is looked up with the device current, once per device
// and context (on every call if the driver cannot give the context's id).
static int noalloc_scratch_address(void** out) {
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return set_error(BSPAI_ERR_UNSUPPORTED, "bspai_gmres_noalloc: device ordinal %d", dev);
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);  // false too while no context is current yet
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    NoallocAddr& a = g_noalloc_base[dev];
    if (!have_id || !a.base || a.ctx_id != id) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(no-allocation scratch)", __FILE__, __LINE__);
        a.base = p;
        unsigned long long id2 = 0;  // the lookup made the device's context current
        a.ctx_id = current_context_id(&id2) ? id2 : 0;
    }
    *out = a.base;
    return BSPAI_OK;
}

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace bspai

extern "C" {

int bspai_gmres_noalloc(bspai_A_h A, bspai_BM_h BM, const double* r, bspai_prec_t u_g, bspai_prec_t u_p,
                        const bspai_opts_t* opts, double* d, bspai_stream_t st, bspai_solve_info_t* info) {
    cudaStream_t s = (cudaStream_t)st;
    if (!A || A->magic != kMagicA) return set_error(BSPAI_ERR_INVALID, "bspai_gmres_noalloc: bad A handle");
    if (!BM || BM->magic != kMagicBM) return set_error(BSPAI_ERR_INVALID, "bspai_gmres_noalloc: bad M handle");
    if (BM->n != A->n) return set_error(BSPAI_ERR_INVALID, "bspai_gmres_noalloc: size mismatch");
    if (A->n > 0 && (!r || !d)) return set_error(BSPAI_ERR_INVALID, "bspai_gmres_noalloc: null vector");
    BSPAI_TRY(check_solver_precs(BSPAI_FP64, BSPAI_DD, u_g, u_p));
    bspai_opts_t o;
    bspai_opts_default(&o);
    if (opts) o = *opts;
    bspai_solve_info_t inf;
    memset(&inf, 0, sizeof inf);
    if (A->n == 0) {
        if (info) *info = inf;
        return BSPAI_OK;
    }
    // workspace layout inside the fixed scratch block
    GmresWork W;
    W.n = A->n;
    W.kmax = resolve_kmax(&o, A->n);
    W.ug = u_g;
    W.up = u_p;
    W.s = s;
    W.tmo_ns = (unsigned long long)((o.barrier_timeout_s > 0 ? o.barrier_timeout_s : 2.0) * 1e9);
    const size_t es = u_g == BSPAI_FP64 ? 8 : 4;
    W.ldv = ceil_div(W.n, 64) * 64;
    int occ = 0, occ2 = 0;
    cudaError_t e = u_g == BSPAI_FP64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mgs<double>, 512, 0)
                                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mgs<float>, 512, 0);
    if (!e)
        e = u_g == BSPAI_FP64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_gmres_start<double>, 512, 0)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_gmres_start<float>, 512, 0);
    if (e) return cuda_error(e, "occupancy", __FILE__, __LINE__);
    occ = occ < occ2 ? occ : occ2;
    if (occ < 1) return set_error(BSPAI_ERR_CUDA, "bspai_gmres_noalloc: cooperative kernel does not fit on an SM");
    W.sms = o.max_blocks > 0 && o.max_blocks < num_sms() ? o.max_blocks : num_sms();
    W.G = (occ >= 2 ? 2 : 1) * W.sms;
    const size_t kx = (size_t)W.kmax;
    size_t off[12];
    size_t sz[11] = {es * (size_t)W.ldv * (kx + 1), es * (size_t)W.ldv, es * 2 * (size_t)W.G, sizeof(GmresState),
                     sizeof(double) * (kx + 1) * kx, sizeof(double) * (kx + 1), sizeof(double) * (kx + 1),
                     sizeof(double) * (kx + 2), sizeof(double) * (kx + 1), sizeof(double) * 4,
                     sizeof(unsigned long long) * GmresWork::tag_words()};
    off[0] = 0;
    for (int i = 0; i < 11; ++i) off[i + 1] = align256(off[i] + sz[i]);
    if (off[11] > kNoallocScratchBytes)
        return set_error(BSPAI_ERR_INVALID,
                         "bspai_gmres_noalloc: n = %d with kmax = %d needs %zu bytes of scratch; the fixed block "
                         "holds %zu bytes (lower kmax or use bspai_gmres)",
                         W.n, W.kmax, off[11], kNoallocScratchBytes);
    unsigned char* base = nullptr;
    BSPAI_TRY(noalloc_scratch_address(reinterpret_cast<void**>(&base)));
    W.V = base + off[0];
    W.w = base + off[1];
    W.part = base + off[2];
    W.st = reinterpret_cast<GmresState*>(base + off[3]);
    W.H = reinterpret_cast<double*>(base + off[4]);
    W.cs = reinterpret_cast<double*>(base + off[5]);
    W.sn = reinterpret_cast<double*>(base + off[6]);
    W.g = reinterpret_cast<double*>(base + off[7]);
    W.y = reinterpret_cast<double*>(base + off[8]);
    W.norms = reinterpret_cast<double*>(base + off[9]);
    W.tags = reinterpret_cast<unsigned long long*>(base + off[10]);
    static thread_local HostFlags t_flags;  // ordinary host memory
    W.hflags = &t_flags;
    BSPAI_TRY(choose_mgs(W));
    // the scratch keeps whatever the previous call left there: clear the parts
    // that must start at zero (solver state with its grid barrier, g, the
    // tagged slots that the barrier's sequence numbers restart with)
    CUDA_TRY(cudaMemsetAsync(W.st, 0, sizeof(GmresState), s));
    CUDA_TRY(cudaMemsetAsync(W.tags, 0, sizeof(unsigned long long) * GmresWork::tag_words(), s));
    CUDA_TRY(cudaMemsetAsync(W.g, 0, sizeof(double) * (kx + 2), s));
    GmresResult gr;
    int rc = u_g == BSPAI_FP64 ? gmres_run<double>(W, A, BM, r, o.tau, nullptr, d, gr)
                               : gmres_run<float>(W, A, BM, r, o.tau, nullptr, d, gr);
    inf.status = rc ? rc : gr.status;
    inf.ir_steps = 1;
    inf.gmres_iters[0] = gr.k;
    inf.total_iters = gr.k;
    inf.relres[0] = gr.beta > 0 ? gr.res / gr.beta : 0.0;
    if (info) *info = inf;
    if (!rc && gr.status == BSPAI_NONFINITE) return set_error(BSPAI_NONFINITE, "bspai_gmres_noalloc: non-finite value");
    return rc;
}

}  // extern "C"
