// batch.cu -- BSPAI-GMRES-IR for many independent systems and right-hand
// sides at once (the batching extension).
//
// Layout: the nsys systems are stacked block-diagonally in one A, one pattern
// and one M (each system padded to a multiple of 32 rows with empty rows), so
// the SPAI build (bspai_build) and the per-system bucketing
// (bspai_bucket_batched) run as single launches over the whole batch.
// Right-hand sides and solutions are nrhs vectors of length n stored one after
// another.  A (system, right-hand side) pair is independent of every other, so
// the GMRES of a refinement step is one persistent launch: each CTA takes pairs
// from a queue (largest systems first) and runs the whole left-preconditioned
// MGS-GMRES of that pair on its own -- bucketed M v and A v over the system's
// rows (the same row arithmetic as the single-system kernels), MGS dot products
// as CTA reductions, Givens rotations and the triangular solve in fp64 -- with
// only CTA barriers, no grid-wide synchronisation.  Per-pair residuals and
// stopping tests (Alg 3.1 loop) run as batched kernels between those launches.
// The schedule of the GMRES launch -- CTA size, the MGS load tile, whether z
// sits in shared memory, and the order in which M's buckets are swept -- is
// picked by timing candidates on a short fixed-length GMRES run of the batch
// (cached per batch shape).  Every candidate computes the same bits for a given
// CTA size: the tile and the bucket order move loads and storage, not the
// order of any sum.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "spmv_row.cuh"
#include "tags.cuh"

namespace bspai {

int launch_residual_batch(const bspai_matrix* A, int nrhs, const double* X, const double* Bv, double* R,
                          const int32_t* slice_seg, int nsys, double* prmax, double* pxmax, cudaStream_t s);

template <typename T>
struct BAr;
template <>
struct BAr<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float sqrt(float a) { return __fsqrt_rn(a); }
};
template <>
struct BAr<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double sqrt(double a) { return __dsqrt_rn(a); }
};

// CTA-wide sum, identical in every thread (fixed reduction tree)
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* s_w) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    if (lane == 0) s_w[w] = v;
    __syncthreads();
    if (w == 0) {
        T t = lane < nw ? s_w[lane] : T(0);
        t = warp_sum(t);
        if (lane == 0) s_w[32] = t;
    }
    __syncthreads();
    const T r = s_w[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ double block_max(double v, double* s_w) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) s_w[w] = v;
    __syncthreads();
    if (w == 0) {
        double t = lane < nw ? s_w[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
        if (lane == 0) s_w[32] = t;
    }
    __syncthreads();
    const double r = s_w[32];
    __syncthreads();
    return r;
}

// Givens rotations on column j of H, update of g, tau test (fp64); thread 0
__device__ void givens_pair(int j, int kmax, double hn, double* H, double* cs, double* sn, double* g, double tau,
                            double beta, double* res, int* done) {
    double* __restrict__ hc = H + (int64_t)j * (kmax + 1);
    const double* __restrict__ c_ = cs;
    const double* __restrict__ s_ = sn;
    hc[j + 1] = hn;
    // the previous rotations applied to the new column; the entry each rotation hands
    // to the next stays in a register, so only the running value is a dependent chain
    // (the stored coefficients and column entries are independent loads)
    double carry = j > 0 ? hc[0] : 0.0;
    for (int i = 0; i < j; ++i) {
        const double ci = c_[i], si = s_[i], hi1 = hc[i + 1];
        const double t1 = __dadd_rn(__dmul_rn(ci, carry), __dmul_rn(si, hi1));
        const double t2 = __dadd_rn(__dmul_rn(-si, carry), __dmul_rn(ci, hi1));
        hc[i] = t1;
        carry = t2;
    }
    if (j > 0) hc[j] = carry;
    const double a = hc[j], b = hc[j + 1];
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
    *res = fabs(g[j + 1]);
    const bool fin = isfinite(*res) && isfinite(hn) && isfinite(rr);
    *done = (*res <= __dmul_rn(tau, beta)) || hn == 0.0 || j + 1 >= kmax || !fin;
}

// y[lr] = (M x)_{r0 + lr} for the rows of one system, under a bucket schedule
// (kept out of line: the kernel calls it three times).
//   MS 0, row-fused: the CTA's threads stride over the rows, two rows per
//     thread at a time (lr and lr + blockDim.x: two independent gather chains),
//     each row through every bucket in turn.
//   MS 1, bucket-major: one sweep over the rows per bucket; each row's
//     partial sum (ascending columns, fp64 for an fp64 bucket, fp32 otherwise)
//     is added in fp64 to the row's running sum in ys, so the sums and their
//     order are those of the row-fused form (yi = 0, then yi + p_k for
//     k = 0, 1, ...).  A row has the same owner thread in every sweep, so ys
//     needs no barrier between sweeps.
template <typename XT, typename YT, int MS>
__device__ __noinline__ void rows_apply(const BMDev& M, int r0, int ns, const XT* __restrict__ x, YT* y,
                                        double* __restrict__ ys) {
    const int bd = blockDim.x;
    if (MS) {
        bool first = true;
        for (int k = 0; k < M.q; ++k) {
            const BucketDev& B = M.b[k];
            if (B.prec == BSPAI_DROP) continue;  // dropped entries are not stored
            for (int lr = threadIdx.x; lr < ns; lr += bd) {
                const int64_t r = r0 + lr, sl = r >> 5;
                const int64_t sb = B.sptr[sl];
                const int w = (int)((B.sptr[sl + 1] - sb) >> 5);
                double p;
                switch (B.prec) {
                case BSPAI_FP64: p = row_partial_f64<XT>(B, sb, w, x, r); break;
                case BSPAI_FP32: p = (double)row_partial_f32<BSPAI_FP32, XT>(B, sb, w, x, r); break;
                case BSPAI_FP16: p = (double)row_partial_f32<BSPAI_FP16, XT>(B, sb, w, x, r); break;
                case BSPAI_BF16: p = (double)row_partial_f32<BSPAI_BF16, XT>(B, sb, w, x, r); break;
                default: p = (double)row_partial_f32<BSPAI_E4M3, XT>(B, sb, w, x, r); break;
                }
                ys[lr] = __dadd_rn(first ? 0.0 : ys[lr], p);
            }
            first = false;
        }
        for (int lr = threadIdx.x; lr < ns; lr += bd) y[lr] = from_f64<YT>(first ? 0.0 : ys[lr]);
        return;
    }
    int lr = threadIdx.x;
    for (; lr + bd < ns; lr += 2 * bd) {
        double ya, yb;
        bucketed_row2<XT>(M, r0 + lr, r0 + lr + bd, x, ya, yb);
        y[lr] = from_f64<YT>(ya);
        y[lr + bd] = from_f64<YT>(yb);
    }
    if (lr < ns) y[lr] = from_f64<YT>(bucketed_row<XT>(M, r0 + lr, x));
}

// The MGS load tile: rows per thread whose loads a pass issues together (two
// candidates per u_g for the autotuner)
template <typename T>
struct MgsU {
    static constexpr int lo = sizeof(T) == 4 ? 8 : 4;
    static constexpr int hi = 2 * lo;
};

struct PairState {
    int32_t* status;   // 0 active; 1 nbe <= u; 2 ||d|| <= u ||x||; 3 stagnation; -1 non-finite
    int32_t* iters;    // GMRES steps summed over refinement steps
    int32_t* steps;    // refinement steps that ran GMRES
    double* rmax;      // per step: max |r| of the pair
    double* xmax;      // per step: max |x| before the update
    double* bmax;      // max |b|
    double* anorm;     // per system ||A_s||_inf
    double* dmax;      // per step: max |d|
    double* dxmax;     // per step: max |x| after the update
    double* dprev;     // previous step's max |d|
    double* relres;    // last GMRES |g_k| / beta
    double* nbe;       // last normwise backward error
};

// U: the MGS load tile.  zcap: pairs of at most zcap rows keep z (the vector
// being orthogonalised) in dynamic shared memory for the whole Arnoldi step
// instead of in its basis slot, which takes the z load and store of every MGS
// pass off the memory system; v_{j+1} is written to the basis once, at the
// end.  MS: the bucket schedule of the M products.
template <typename T, int U, int MS>
__global__ void __launch_bounds__(512, 1) k_gmres_batch(const __grid_constant__ BMDev Av, const __grid_constant__ BMDev Mv,
                                                      const int32_t* __restrict__ row_off, int nsys, int n,
                                                      const int32_t* __restrict__ order, int npairs, int* queue,
                                                      const int32_t* __restrict__ status, const double* __restrict__ R,
                                                      double* __restrict__ X, T* Vws, T* Wws, double* Yws, int64_t ldv,
                                                      double* Hws, double* Sws, int kmax, double tau, int zcap,
                                                      int32_t* __restrict__ iters,
                                                      int32_t* __restrict__ steps, double* __restrict__ relres,
                                                      double* __restrict__ dmax, double* __restrict__ dxmax,
                                                      unsigned long long* __restrict__ work) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    T* const s_z = reinterpret_cast<T*>(s_dyn);
    __shared__ T s_w[33];
    __shared__ double s_d[33];
    __shared__ int s_p, s_done;
    __shared__ double s_res;
    using Ar = BAr<T>;
    const int tid = threadIdx.x, bd = blockDim.x;
    T* V = Vws + (int64_t)blockIdx.x * ldv * (kmax + 1);
    T* w = Wws + (int64_t)blockIdx.x * ldv;
    double* H = Hws + (int64_t)blockIdx.x * (kmax + 1) * kmax;
    double* cs = Sws + (int64_t)blockIdx.x * 4 * (kmax + 2);
    double* sn = cs + (kmax + 2);
    double* g = sn + (kmax + 2);
    double* y = g + (kmax + 2);
    while (true) {
        if (tid == 0) s_p = atomicAdd(queue, 1);
        __syncthreads();
        const int p = s_p;
        __syncthreads();
        if (p >= npairs) break;
        const int pair = order[p];
        if (status[pair] != 0) continue;
        const int rhs = pair / nsys, sys = pair - rhs * nsys;
        const int r0 = row_off[sys], ns = row_off[sys + 1] - r0;
        const double* rr = R + (int64_t)rhs * n;
        double* xx = X + (int64_t)rhs * n;
        // s = M r (Alg 2.3), stored in u_g; beta = ||s||_2
        rows_apply<double, T, MS>(Mv, r0, ns, rr, V, Yws + (int64_t)blockIdx.x * ldv);
        T acc = T(0);
        for (int lr = tid; lr < ns; lr += bd) acc = Ar::add(acc, Ar::mul(V[lr], V[lr]));
        const T beta = Ar::sqrt(block_sum(acc, s_w));
        const bool fin = isfinite((double)beta);
        int k = 0;
        double res = (double)beta;
        if (beta > T(0) && fin) {
            for (int lr = tid; lr < ns; lr += bd) V[lr] = Ar::div(V[lr], beta);
            if (tid == 0) g[0] = (double)beta;
            for (int j = 0; j < kmax; ++j) {
                __syncthreads();
                const T* vj = V + (int64_t)j * ldv;
                rows_apply<T, T, 0>(Av, r0, ns, vj - r0, w, nullptr);
                __syncthreads();
                T* z = ns <= zcap ? s_z : V + (int64_t)(j + 1) * ldv;
                rows_apply<T, T, MS>(Mv, r0, ns, w - r0, z, Yws + (int64_t)blockIdx.x * ldv);
                // modified Gram-Schmidt: pass i updates z by the previous coefficient and
                // dots it with v_i; the last pass forms ||z||_2 (each thread owns its rows of z)
                T hprev = T(0);
                for (int i = 0; i <= j + 1; ++i) {
                    const T* vi = V + (int64_t)(i <= j ? i : j) * ldv;
                    const T* vp = V + (int64_t)(i > 0 ? i - 1 : 0) * ldv;
                    T a = T(0);
                    // U rows of the thread at a time, all their loads issued before
                    // any store (z shares V's storage, so without this every load
                    // would wait for the previous row's store); the rows are still
                    // accumulated in the order tid, tid + bd, tid + 2 bd, ...
                    for (int b0 = tid; b0 < ns; b0 += bd * U) {
                        T zr[U], pv[U], iv[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int lr = b0 + u * bd;
                            if (lr < ns) {
                                zr[u] = z[lr];
                                pv[u] = i > 0 ? vp[lr] : T(0);
                                iv[u] = i <= j ? vi[lr] : T(0);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int lr = b0 + u * bd;
                            if (lr < ns) {
                                if (i > 0) {
                                    zr[u] = Ar::sub(zr[u], Ar::mul(hprev, pv[u]));
                                    z[lr] = zr[u];
                                }
                                a = Ar::add(a, Ar::mul(i <= j ? iv[u] : zr[u], zr[u]));
                            }
                        }
                    }
                    const T h = block_sum(a, s_w);
                    if (i <= j) {
                        if (tid == 0) H[(int64_t)j * (kmax + 1) + i] = (double)h;
                        hprev = h;
                    } else {
                        const T hn = Ar::sqrt(h);
                        // v_{j+1} = z / h_{j+1,j} into the basis (in place when z lives there)
                        const bool nz = hn > T(0) && isfinite((double)hn);
                        T* vn = V + (int64_t)(j + 1) * ldv;
                        if (nz || vn != z)
                            for (int lr = tid; lr < ns; lr += bd) vn[lr] = nz ? Ar::div(z[lr], hn) : z[lr];
                        if (tid == 0) {
                            double rs;
                            int dn;
                            givens_pair(j, kmax, (double)hn, H, cs, sn, g, tau, (double)beta, &rs, &dn);
                            s_res = rs;
                            s_done = dn;
                        }
                    }
                }
                __syncthreads();
                if (tid == 0 && work) {  // rows read by the j + 2 passes, rows of the step's products
                    atomicAdd(work, (unsigned long long)(j + 2) * (unsigned long long)ns);
                    atomicAdd(work + 1, (unsigned long long)ns);
                }
                k = j + 1;
                res = s_res;
                if (s_done) break;
            }
            // y = R^-1 g, column-oriented back substitution (fp64)
            __syncthreads();
            for (int i = k - 1; i >= 0; --i) {
                const double* hc = H + (int64_t)i * (kmax + 1);
                if (tid == 0) y[i] = __ddiv_rn(g[i], hc[i]);
                __syncthreads();
                const double yi = y[i];
                for (int t = tid; t < i; t += bd) g[t] = __dsub_rn(g[t], __dmul_rn(hc[t], yi));
                __syncthreads();
            }
        }
        // d = V y in u_g, x += d in fp64
        double dm = 0.0, xm = 0.0;
        for (int lr = tid; lr < ns; lr += bd) {
            T a = T(0);
            for (int jj = 0; jj < k; ++jj) a = Ar::add(a, Ar::mul(V[(int64_t)jj * ldv + lr], from_f64<T>(y[jj])));
            const double d = (double)a;
            const double xn = __dadd_rn(xx[r0 + lr], d);
            xx[r0 + lr] = xn;
            double ad = fabs(d), ax = fabs(xn);
            if (!(ad <= 1.7976931348623157e308)) ad = __longlong_as_double(0x7ff0000000000000LL);
            if (!(ax <= 1.7976931348623157e308)) ax = __longlong_as_double(0x7ff0000000000000LL);
            dm = fmax(dm, ad);
            xm = fmax(xm, ax);
        }
        dm = block_max(dm, s_d);
        xm = block_max(xm, s_d);
        if (tid == 0) {
            iters[pair] += k;
            steps[pair] += 1;
            relres[pair] = beta > T(0) ? res / (double)beta : 0.0;
            dmax[pair] = fin ? dm : __longlong_as_double(0x7ff0000000000000LL);
            dxmax[pair] = xm;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ teams
// Team mode (u_g = fp32): a pair of n_s rows runs on a team of
// G = ceil(n_s / team_rows) CTAs of one cooperative launch, each CTA owning a
// contiguous chunk of the pair's rows.  As in the single-system on-chip MGS
// kernel, z and the basis rows of the current and next pass stay in registers
// (row pairs, packed two-lane arithmetic), so an MGS pass reads each basis row
// once; the j + 2 reductions of an Arnoldi step, and the barriers between the
// products (A v_j reads every rank's rows of v_j, M w every rank's rows of w),
// are tagged-slot exchanges among the team's CTAs with bounded waits.  Data
// another CTA of the launch wrote is read from L2 (ld.global.cg), after a
// release/acquire pair of fences around the exchange.  The dot products sum a
// thread's rows, then the CTA in a fixed tree, then the team's CTAs in rank
// order: the same in every CTA and every run, but another order than the
// one-CTA schedules (so other bits, within the same parity bars).
constexpr int kTeamBD = 512;   // threads of a team CTA
constexpr int kTeamP = 8;      // row pairs per thread: at most 8,192 rows of a pair per CTA
                               // (16 pairs, as the single-system kernel holds, spill registers here)
constexpr int kTeamMaxG = 32;  // CTAs of one team (one polling lane each)

// One group of the launch: the pairs of one team size (a run of the
// size-sorted order) and the CTAs given to them, with the group's share of the
// workspace
struct TeamGroup {
    int G;        // CTAs per team
    int begin;    // first pair of the run in the order
    int count;    // its pairs
    int cta0;     // first CTA of the group
    int nteams;   // its teams
    int64_t ldv;  // rows of a vector (largest system of the run, rounded up to 64)
    int64_t voff, woff, hoff, soff, toff;  // the group's first team in V, W / Z, H, S, tags
};
constexpr int kTeamMaxGroups = 32;

struct TeamArgs {
    BMDev Av, Mv;
    const int32_t* row_off;
    int nsys, n;
    const int32_t* order;  // the size-sorted pairs (each group takes a run)
    int* queue;            // one per group
    const int32_t* status;
    const double* R;
    double* X;
    float* V;  // per team: ldv x (kmax + 1)
    float* W;  // per team: ldv (A v)
    float* Z;  // per team: ldv (s = M r, then M w)
    double* H;  // per team: (kmax + 1) x kmax
    double* S;  // per team: cs, sn, g, y (kmax + 2 each)
    int kmax;
    double tau;
    int ngroups;
    TeamGroup grp[kTeamMaxGroups];
    unsigned long long* tags;  // per team: 2 sets x G slots x 2 words
    GridBar* bar;              // err: a team exchange timed out
    unsigned long long tmo;
    int32_t *iters, *steps;
    double *relres, *dmax, *dxmax;
    unsigned long long* work;  // [0] rows read by MGS passes, [1] rows of the Arnoldi steps' products
};

struct TeamSync {
    unsigned long long* tags;
    GridBar* bar;
    unsigned long long tmo;
    int G, rank;
    unsigned seq;  // exchanges so far: the same count in every CTA of the team
};

__device__ __forceinline__ float warp_max_nn(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max_nn(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <int OP, typename T>
__device__ __forceinline__ T warp_comb(T v) {
    if constexpr (OP == 0) return warp_sum(v);
    else return warp_max_nn(v);
}

// First half of a team exchange: the CTA's threads' values combined (OP 0: a
// sum in a fixed tree; OP 1: a max of non-negative values) and published in
// the CTA's slot.  FENCE: the CTA's earlier writes are released with it.
template <typename T, int OP, bool FENCE>
__device__ __forceinline__ void team_arrive(TeamSync& ts, T v, T* s_w, T* s_tot) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_comb<OP>(v);
    if (lane == 0) s_w[w] = v;
    __syncthreads();
    ts.seq += 1u;
    if (w == 0) {
        T t = lane < nw ? s_w[lane] : T(0);
        t = warp_comb<OP>(t);
        if (lane == 0) {
            if (ts.G == 1) {
                *s_tot = t;
            } else {
                if (FENCE) __threadfence();
                tag_publish(t, ts.tags + (int64_t)(ts.seq & 1u) * 2 * ts.G + (int64_t)ts.rank * TagWords<T>::W,
                            ts.seq);
            }
        }
    }
}

// Second half: warp 0 polls the team's slots until all carry this exchange's
// number (giving up after tmo ns, or once any CTA of the launch has flagged an
// error), combines them in rank order, and every thread gets the result.
// *s_ok = 0 after a timeout.  FENCE: the other CTAs' released writes are
// visible to this CTA's threads after it.
template <typename T, int OP, bool FENCE>
__device__ __forceinline__ T team_wait(TeamSync& ts, T* s_tot, int* s_ok) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        bool ok = true;
        if (ts.G > 1) {
            const unsigned long long* base = ts.tags + (int64_t)(ts.seq & 1u) * 2 * ts.G;
            T val = T(0);
            bool have = lane >= ts.G;
            unsigned long long t0 = 0;
            for (int it = 0;; ++it) {
                if (!have) have = tag_read(base + (int64_t)lane * TagWords<T>::W, ts.seq, &val);
                if (__all_sync(0xffffffffu, have)) break;
                int stop = 0;
                if (lane == 0) {
                    const unsigned long long now = globaltimer_ns();
                    if (it == 0) t0 = now;
                    if (now - t0 > ts.tmo) {
                        atomicExch(&ts.bar->err, 1);
                        stop = 1;
                    } else if ((it & 63) == 63 && *(volatile int*)&ts.bar->err) {
                        stop = 1;
                    }
                }
                if (__shfl_sync(0xffffffffu, stop, 0)) {
                    ok = false;
                    break;
                }
            }
            const T t = warp_comb<OP>(val);
            if (FENCE) __threadfence();
            if (lane == 0) *s_tot = t;
        }
        if (lane == 0) *s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    return *s_tot;
}

// y[lr] = (M x)_{r0 + lr} in u_g for the rows lo .. hi - 1 of one pair, two
// rows per thread at a time (as rows_apply); CG: x is read from L2
template <typename XT, bool CG>
__device__ __noinline__ void team_rows(const BMDev& M, int r0, int lo, int hi, const XT* __restrict__ x, float* y) {
    const int bd = blockDim.x;
    int lr = lo + threadIdx.x;
    for (; lr + bd < hi; lr += 2 * bd) {
        double ya, yb;
        bucketed_row2<XT, CG>(M, r0 + lr, r0 + lr + bd, x, ya, yb);
        y[lr] = from_f64<float>(ya);
        y[lr + bd] = from_f64<float>(yb);
    }
    if (lr < hi) y[lr] = from_f64<float>(bucketed_row<XT, CG>(M, r0 + lr, x));
}

__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

// The modified Gram-Schmidt passes of Arnoldi step j for one CTA of a team (z
// from this CTA's rows of Z, the basis rows in registers; H column j written by
// rank 0) and v_{j+1} = z / h_{j+1,j} into the basis; returns h_{j+1,j}.
// Out of line, so that the register arrays of the passes have the kernel's
// whole register budget.  *s_ok = 0 after a timed-out exchange.
template <int P>
__device__ __noinline__ float team_mgs(float* V, int64_t ldv, const float* Z, int lo, int nb, int j, int kmax,
                                       double* H, TeamSync& ts, float* s_wf, float* s_totf, int* s_ok) {
    constexpr int BD = kTeamBD;
    const int tid = threadIdx.x, rank = ts.rank;
    const float2 zero2 = make_float2(0.0f, 0.0f);
    // this CTA's rows: pair q = tid + s BD covers rows lo + 2q, lo + 2q + 1
    auto ld2 = [&](const float* base, int q) -> float2 {
        const float* p2 = base + lo + 2 * q;
        if (2 * q + 1 < nb) return __ldcg(reinterpret_cast<const float2*>(p2));
        return make_float2(__ldcg(p2), 0.0f);
    };
    float2 zr[P], vcur[P], vnext[P];
    // modified Gram-Schmidt: pass i takes z -= h_{i-1} v_{i-1} and dots z with v_i
    // (the last pass forms ||z||^2), the loads of v_i issued before the wait
    float2 acc2 = zero2;
#pragma unroll
    for (int t = 0; t < P; ++t) {
        const int q = tid + t * BD;
        zr[t] = zero2;
        vcur[t] = zero2;
        vnext[t] = zero2;
        if (2 * q < nb) {
            zr[t] = ld2(Z, q);
            vcur[t] = ld2(V, q);
            acc2 = __fadd2_rn(acc2, __fmul2_rn(vcur[t], zr[t]));
        }
    }
    team_arrive<float, 0, false>(ts, __fadd_rn(acc2.x, acc2.y), s_wf, s_totf);
    for (int i = 1; i <= j + 1; ++i) {
        if (i <= j) {
            const float* vi = V + (int64_t)i * ldv;
#pragma unroll
            for (int t = 0; t < P; ++t) {
                const int q = tid + t * BD;
                if (2 * q < nb) vnext[t] = ld2(vi, q);
            }
        }
        const float h = team_wait<float, 0, false>(ts, s_totf, s_ok);
        if (!*s_ok) return 0.0f;
        if (rank == 0 && tid == 0) H[(int64_t)j * (kmax + 1) + (i - 1)] = (double)h;
        const float2 h2 = make_float2(h, h);
        acc2 = zero2;
#pragma unroll
        for (int t = 0; t < P; ++t) {
            const int q = tid + t * BD;
            if (2 * q < nb) {
                zr[t] = f2sub(zr[t], __fmul2_rn(h2, vcur[t]));
                acc2 = __fadd2_rn(acc2, __fmul2_rn(i <= j ? vnext[t] : zr[t], zr[t]));
            }
        }
        team_arrive<float, 0, false>(ts, __fadd_rn(acc2.x, acc2.y), s_wf, s_totf);
#pragma unroll
        for (int t = 0; t < P; ++t) vcur[t] = vnext[t];
    }
    const float hz = team_wait<float, 0, false>(ts, s_totf, s_ok);
    if (!*s_ok) return 0.0f;
    const float hn = __fsqrt_rn(hz);
    const bool norm = hn > 0.0f && isfinite((double)hn);
    float* vn = V + (int64_t)(j + 1) * ldv + lo;
#pragma unroll
    for (int t = 0; t < P; ++t) {
        const int q = tid + t * BD;
        if (2 * q < nb) {
            float2 zo = zr[t];
            if (norm) zo = make_float2(__fdiv_rn(zo.x, hn), __fdiv_rn(zo.y, hn));
            if (2 * q + 1 < nb) *reinterpret_cast<float2*>(vn + 2 * q) = zo;
            else vn[2 * q] = zo.x;
        }
    }
    return hn;
}

template <int P>
__global__ void __launch_bounds__(kTeamBD, 1) k_gmres_team(const __grid_constant__ TeamArgs a) {
    constexpr int BD = kTeamBD;
    extern __shared__ float s_y[];  // y of the pair in u_g (kmax entries)
    __shared__ float s_wf[32];
    __shared__ double s_wd[32];
    __shared__ float s_totf;
    __shared__ double s_totd;
    __shared__ int s_ok, s_p, s_done;
    __shared__ double s_res;
    const int tid = threadIdx.x;
    // this CTA's group, team and rank
    int gi = 0;
    while (gi + 1 < a.ngroups && (int)blockIdx.x >= a.grp[gi + 1].cta0) ++gi;
    const TeamGroup& gr = a.grp[gi];
    const int G = gr.G;
    const int local = (int)blockIdx.x - gr.cta0;
    if (local >= gr.nteams * G) return;  // (a CTA past the groups' teams: none is launched)
    const int team = local / G, rank = local - team * G;
    const int kmax = a.kmax;
    const int64_t ldv = gr.ldv;
    float* V = a.V + gr.voff + (int64_t)team * ldv * (kmax + 1);
    float* W = a.W + gr.woff + (int64_t)team * ldv;
    float* Z = a.Z + gr.woff + (int64_t)team * ldv;
    double* H = a.H + gr.hoff + (int64_t)team * (kmax + 1) * kmax;
    double* cs = a.S + gr.soff + (int64_t)team * 4 * (kmax + 2);
    double* sn = cs + (kmax + 2);
    double* g = sn + (kmax + 2);
    double* y = g + (kmax + 2);
    TeamSync ts{a.tags + gr.toff + (int64_t)team * 4 * G, a.bar, a.tmo, G, rank, 0u};
    const float2 zero2 = make_float2(0.0f, 0.0f);
    // the team's own group first, then (its queue empty) the groups of smaller pairs:
    // their systems fit the team's workspace and its CTAs, and no team idles while
    // pairs are left
    int qg = gi;
    while (true) {
        // the next pair: rank 0 takes it from the queue, the team learns it by an exchange
        if (rank == 0 && tid == 0) s_p = atomicAdd(a.queue + qg, 1);
        __syncthreads();
        team_arrive<float, 0, false>(ts, (rank == 0 && tid == 0) ? (float)s_p : 0.0f, s_wf, &s_totf);
        const int p = (int)team_wait<float, 0, false>(ts, &s_totf, &s_ok);
        if (!s_ok) return;
        if (p >= a.grp[qg].count) {
            if (++qg >= a.ngroups) return;
            continue;
        }
        const int pair = a.order[a.grp[qg].begin + p];
        if (a.status[pair] != 0) continue;
        const int rhs = pair / a.nsys, sys = pair - rhs * a.nsys;
        const int r0 = a.row_off[sys], ns = a.row_off[sys + 1] - r0;
        const double* rr = a.R + (int64_t)rhs * a.n;
        double* xx = a.X + (int64_t)rhs * a.n;
        const int chunk = (int)(ceil_div(ceil_div(ns, G), 64) * 64);
        const int lo = rank * chunk < ns ? rank * chunk : ns;
        const int hi = lo + chunk < ns ? lo + chunk : ns;
        const int nb = hi - lo;
        // this CTA's rows: pair q = tid + s BD covers rows lo + 2q, lo + 2q + 1
        auto ld2 = [&](const float* base, int q) -> float2 {
            const float* p2 = base + lo + 2 * q;
            if (2 * q + 1 < nb) return __ldcg(reinterpret_cast<const float2*>(p2));
            return make_float2(__ldcg(p2), 0.0f);
        };
        auto st2 = [&](float* base, int q, float2 v) {
            float* p2 = base + lo + 2 * q;
            if (2 * q + 1 < nb) *reinterpret_cast<float2*>(p2) = v;
            else *p2 = v.x;
        };
        float2 zr[P];
        // s = M r (Alg 2.3) in u_g; beta = ||s||_2
        team_rows<double, false>(a.Mv, r0, lo, hi, rr, Z);
        __syncthreads();
        float2 acc2 = zero2;
#pragma unroll
        for (int t = 0; t < P; ++t) {
            const int q = tid + t * BD;
            zr[t] = zero2;
            if (2 * q < nb) {
                zr[t] = ld2(Z, q);
                acc2 = __fadd2_rn(acc2, __fmul2_rn(zr[t], zr[t]));
            }
        }
        team_arrive<float, 0, false>(ts, __fadd_rn(acc2.x, acc2.y), s_wf, &s_totf);
        const float beta = __fsqrt_rn(team_wait<float, 0, false>(ts, &s_totf, &s_ok));
        if (!s_ok) return;
        const bool fin = isfinite((double)beta);
        int k = 0;
        double res = (double)beta;
        if (beta > 0.0f && fin) {
#pragma unroll
            for (int t = 0; t < P; ++t) {
                const int q = tid + t * BD;
                if (2 * q < nb) st2(V, q, make_float2(__fdiv_rn(zr[t].x, beta), __fdiv_rn(zr[t].y, beta)));
            }
            if (rank == 0 && tid == 0) g[0] = (double)beta;
            for (int j = 0; j < kmax; ++j) {
                // barrier: v_j complete in every rank
                __syncthreads();
                team_arrive<float, 0, true>(ts, 0.0f, s_wf, &s_totf);
                team_wait<float, 0, true>(ts, &s_totf, &s_ok);
                if (!s_ok) return;
                const float* vj = V + (int64_t)j * ldv;
                team_rows<float, true>(a.Av, r0, lo, hi, vj - r0, W);
                __syncthreads();
                team_arrive<float, 0, true>(ts, 0.0f, s_wf, &s_totf);
                team_wait<float, 0, true>(ts, &s_totf, &s_ok);
                if (!s_ok) return;
                team_rows<float, true>(a.Mv, r0, lo, hi, W - r0, Z);
                __syncthreads();
                const float hn = team_mgs<P>(V, ldv, Z, lo, nb, j, kmax, H, ts, s_wf, &s_totf, &s_ok);
                if (!s_ok) return;
                if (rank == 0 && tid == 0) {
                    double rs;
                    int dn;
                    givens_pair(j, kmax, (double)hn, H, cs, sn, g, a.tau, (double)beta, &rs, &dn);
                    s_res = rs;
                    s_done = dn;
                }
                __syncthreads();
                // every rank learns rank 0's stopping decision (the next barrier is the loop's)
                team_arrive<float, 0, false>(ts, (rank == 0 && tid == 0) ? (float)s_done : 0.0f, s_wf, &s_totf);
                const float dn = team_wait<float, 0, false>(ts, &s_totf, &s_ok);
                if (!s_ok) return;
                if (rank == 0 && tid == 0 && a.work) {
                    atomicAdd(a.work, (unsigned long long)(j + 2) * (unsigned long long)ns);
                    atomicAdd(a.work + 1, (unsigned long long)ns);
                }
                k = j + 1;
                if (rank == 0) res = s_res;
                if (dn != 0.0f) break;
            }
            // y = R^-1 g, column-oriented back substitution (fp64, rank 0)
            if (rank == 0) {
                __syncthreads();
                for (int i = k - 1; i >= 0; --i) {
                    const double* hc = H + (int64_t)i * (kmax + 1);
                    if (tid == 0) y[i] = __ddiv_rn(g[i], hc[i]);
                    __syncthreads();
                    const double yi = y[i];
                    for (int t = tid; t < i; t += BD) g[t] = __dsub_rn(g[t], __dmul_rn(hc[t], yi));
                    __syncthreads();
                }
            }
            __syncthreads();
            team_arrive<float, 0, true>(ts, 0.0f, s_wf, &s_totf);
            team_wait<float, 0, true>(ts, &s_totf, &s_ok);
            if (!s_ok) return;
            for (int t = tid; t < k; t += BD) s_y[t] = from_f64<float>(__ldcg(y + t));
            __syncthreads();
        }
        // d = V y in u_g, x += d in fp64 (this CTA's rows)
        double dm = 0.0, xm = 0.0;
        for (int lr = lo + tid; lr < hi; lr += BD) {
            float acc = 0.0f;
            for (int jj = 0; jj < k; ++jj) acc = __fadd_rn(acc, __fmul_rn(__ldcg(V + (int64_t)jj * ldv + lr), s_y[jj]));
            const double d = (double)acc;
            const double xn = __dadd_rn(xx[r0 + lr], d);
            xx[r0 + lr] = xn;
            double ad = fabs(d), ax = fabs(xn);
            if (!(ad <= 1.7976931348623157e308)) ad = __longlong_as_double(0x7ff0000000000000LL);
            if (!(ax <= 1.7976931348623157e308)) ax = __longlong_as_double(0x7ff0000000000000LL);
            dm = fmax(dm, ad);
            xm = fmax(xm, ax);
        }
        team_arrive<double, 1, false>(ts, dm, s_wd, &s_totd);
        dm = team_wait<double, 1, false>(ts, &s_totd, &s_ok);
        if (!s_ok) return;
        team_arrive<double, 1, false>(ts, xm, s_wd, &s_totd);
        xm = team_wait<double, 1, false>(ts, &s_totd, &s_ok);
        if (!s_ok) return;
        if (rank == 0 && tid == 0) {
            a.iters[pair] += k;
            a.steps[pair] += 1;
            a.relres[pair] = beta > 0.0f ? res / (double)beta : 0.0;
            a.dmax[pair] = fin ? dm : __longlong_as_double(0x7ff0000000000000LL);
            a.dxmax[pair] = xm;
        }
        __syncthreads();
    }
}

// per pair: nbe = ||r|| / (||A_s|| ||x|| + ||b||); stop when <= u; count active pairs
__global__ void k_batch_flags(int npairs, int nsys, PairState S, double ustop, int* active) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    if (S.status[p] != 0) return;
    const double rm = S.rmax[p];
    const double den = S.anorm[p % nsys] * S.xmax[p] + S.bmax[p];
    const double nbe = rm == 0.0 ? 0.0 : rm / den;
    S.nbe[p] = nbe;
    if (!isfinite(nbe)) {
        S.status[p] = -1;
        return;
    }
    if (nbe <= ustop) {
        S.status[p] = 1;
        return;
    }
    atomicAdd(active, 1);
}

// per pair after the update: ||d|| <= u ||x||, or stagnation ||d_i|| > stag ||d_{i-1}||
__global__ void k_batch_after(int npairs, PairState S, double ustop, double stag) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    if (S.status[p] != 0) return;
    const double d = S.dmax[p], xm = S.dxmax[p];
    if (!isfinite(d) || !isfinite(xm)) {
        S.status[p] = -1;
        return;
    }
    if (d <= __dmul_rn(ustop, xm)) S.status[p] = 2;
    else if (d > __dmul_rn(stag, S.dprev[p])) S.status[p] = 3;
    S.dprev[p] = d;
}

__global__ void k_system_norms(int n, const int64_t* __restrict__ sptr, const int32_t* __restrict__ col,
                               const double* __restrict__ val, const int32_t* __restrict__ slice_seg,
                               double* __restrict__ anorm) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double sum = 0.0;
    if (r < n)
        for (int64_t p = sptr[r >> 5] + (r & 31); p < sptr[(r >> 5) + 1]; p += kSlice)
            if (col[p] >= 0) sum = __dadd_rn(sum, fabs(val[p]));
    // one slice per warp, so one system: one atomic per warp
    sum = warp_max_bits(sum);
    if ((threadIdx.x & 31) == 0 && r < n && sum != 0.0) atomic_max_nonneg(anorm + slice_seg[r >> 5], sum);
}

__global__ void k_pair_bmax(int n, int nrhs, int nsys, const double* __restrict__ Bv,
                            const int32_t* __restrict__ slice_seg, double* __restrict__ bmax) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * nrhs) return;
    const int64_t rhs = t / n, i = t - rhs * n;
    double a = fabs(Bv[t]);
    if (!(a <= 1.7976931348623157e308)) a = __longlong_as_double(0x7ff0000000000000LL);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(bmax + rhs * nsys + slice_seg[i >> 5], a);
}

__global__ void k_fill_d(int64_t count, double* __restrict__ p, double v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) p[i] = v;
}

__global__ void k_slice_seg_b(int nsys, const int32_t* __restrict__ row_off, int32_t* __restrict__ slice_seg) {
    const int sg = blockIdx.x * blockDim.x + threadIdx.x;
    if (sg >= nsys) return;
    for (int s = row_off[sg] >> 5; s < (row_off[sg + 1] >> 5); ++s) slice_seg[s] = sg;
}

// ------------------------------------------------------------------ host
struct TuneKey {
    int n, nsys, nrhs, ug, kmax;
    bool operator<(const TuneKey& o) const {
        return std::tie(n, nsys, nrhs, ug, kmax) < std::tie(o.n, o.nsys, o.nrhs, o.ug, o.kmax);
    }
};

// One schedule of the batched GMRES launch (see bspai_batch_schedule_t)
struct Sched {
    int bd = 512;     // CTA size
    int urows = 0;    // MGS load tile (rows per thread), 0: the smaller candidate
    int zcap = 0;     // pairs of at most zcap rows keep z in shared memory
    int msched = 0;   // 0 row-fused, 1 bucket-major
    int team = 0;     // > 0: team mode, rows of a pair per CTA of its team (u_g = fp32)
};

static std::mutex g_tune_mu;
static std::map<TuneKey, Sched> g_tuned;  // schedule per batch shape
static std::vector<bspai_batch_schedule_t> g_table_s;  // the last tuning's candidates, in the order timed
static std::vector<float> g_table_ms;
static thread_local bool t_forced = false;
static thread_local Sched t_force;

template <typename T>
using BatchKernel = decltype(&k_gmres_batch<T, MgsU<T>::lo, 0>);

template <typename T>
static BatchKernel<T> batch_kernel(int urows, int msched) {
    if (urows == MgsU<T>::hi) return msched ? k_gmres_batch<T, MgsU<T>::hi, 1> : k_gmres_batch<T, MgsU<T>::hi, 0>;
    return msched ? k_gmres_batch<T, MgsU<T>::lo, 1> : k_gmres_batch<T, MgsU<T>::lo, 0>;
}

template <typename T>
static int occupancy_blocks(BatchKernel<T> kern, int bd, size_t smem, int* occ) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, bd, smem);
    if (e) return cuda_error(e, "occupancy", __FILE__, __LINE__);
    return BSPAI_OK;
}

// The largest z_shared_rows for this kernel and CTA size that keeps the CTAs per
// SM its registers allow (0 when none fit); raises the kernel's dynamic shared
// memory limit to the opt-in maximum on the way.
template <typename T>
static int zcap_limit(BatchKernel<T> kern, int bd, int* zmax) {
    int dev = 0, sm_bytes = 0, blk_bytes = 0, occ0 = 0;
    cudaFuncAttributes fa;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    CUDA_TRY(cudaDeviceGetAttribute(&blk_bytes, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
    const int dyn_max = blk_bytes - (int)fa.sharedSizeBytes;
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max));
    int rc = occupancy_blocks<T>(kern, bd, 0, &occ0);
    if (rc) return rc;
    *zmax = 0;
    if (occ0 < 1) return BSPAI_OK;
    // 1 KB of shared memory per CTA is reserved by the system
    int bytes = sm_bytes / occ0 - (int)fa.sharedSizeBytes - 1024;
    if (bytes > dyn_max) bytes = dyn_max;
    for (int z = bytes / (int)sizeof(T) / 32 * 32; z >= 32; z -= 256) {
        int occ = 0;
        if ((rc = occupancy_blocks<T>(kern, bd, sizeof(T) * (size_t)z, &occ))) return rc;
        if (occ >= occ0) {
            *zmax = z;
            return BSPAI_OK;
        }
    }
    return BSPAI_OK;
}

template <typename T>
static int batch_ir(bspai_matrix* A, const int32_t* row_off, int nsys, int nrhs, const double* Bv,
                    const bspai_bucketed* BM, const bspai_spai* M, int u_p, double tol, const bspai_opts_t& o,
                    double* X, cudaStream_t s, bspai_batch_info_t* info, int32_t* pair_status, int32_t* pair_iters) {
    const int n = A->n;
    const int npairs = nsys * nrhs;
    const int nsl = A->sell.nslices;
    const int ug = sizeof(T) == 8 ? BSPAI_FP64 : BSPAI_FP32;
    // host copy of the offsets: sizes, ordering, workspace
    std::vector<int32_t> hoff((size_t)nsys + 1);
    CUDA_TRY(cudaMemcpyAsync(hoff.data(), row_off, sizeof(int32_t) * ((size_t)nsys + 1), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (hoff[0] != 0 || hoff[nsys] != n) return set_error(BSPAI_ERR_INVALID, "batched solve: row_off must run from 0 to n");
    int nmax = 0;
    for (int k = 0; k < nsys; ++k) {
        const int len = hoff[k + 1] - hoff[k];
        if (len < 0 || (hoff[k] & 31)) return set_error(BSPAI_ERR_INVALID, "batched solve: offsets must be multiples of 32");
        nmax = len > nmax ? len : nmax;
    }
    int kmax = o.kmax > 0 ? o.kmax : (nmax < 300 ? nmax : 300);
    if (kmax < 1) kmax = 1;
    int imax = o.i_max > 0 ? o.i_max : 10;
    if (imax > 32) imax = 32;
    const double ustop = o.u_stop > 0 ? o.u_stop : 0x1p-53;
    const double stag = o.stagnation > 0 ? o.stagnation : 0.9;
    const double tau = tol > 0 ? tol : o.tau;
    // pairs, largest systems first
    std::vector<int32_t> hord((size_t)npairs);
    {
        std::vector<int32_t> sys(nsys);
        for (int k = 0; k < nsys; ++k) sys[k] = k;
        std::stable_sort(sys.begin(), sys.end(), [&](int a, int b) {
            return (hoff[a + 1] - hoff[a]) > (hoff[b + 1] - hoff[b]);
        });
        size_t c = 0;
        for (int k : sys)
            for (int r = 0; r < nrhs; ++r) hord[c++] = r * nsys + k;
    }
    const int64_t ldv = ceil_div(nmax > 0 ? nmax : 1, 64) * 64;
    // device buffers
    std::vector<void*> bufs;
    auto take = [&](void** p, size_t bytes) {
        int rc = dalloc(p, bytes, s);
        if (!rc) bufs.push_back(*p);
        return rc;
    };
    auto done = [&](int code) {
        for (void* p : bufs) dfree(p, s);
        return code;
    };
    PairState S{};
    int32_t *d_order = nullptr, *d_seg = nullptr, *d_queue = nullptr, *d_active = nullptr;
    double* R = nullptr;
    int rc;
    if ((rc = take((void**)&d_order, sizeof(int32_t) * npairs))) return done(rc);
    if ((rc = take((void**)&d_seg, sizeof(int32_t) * (size_t)(nsl > 0 ? nsl : 1)))) return done(rc);
    if ((rc = take((void**)&d_queue, sizeof(int) * 2))) return done(rc);
    d_active = d_queue + 1;
    if ((rc = take((void**)&R, sizeof(double) * (size_t)n * nrhs))) return done(rc);
    void* p;
    if ((rc = take(&p, sizeof(int32_t) * npairs * 3))) return done(rc);
    S.status = (int32_t*)p;
    S.iters = S.status + npairs;
    S.steps = S.iters + npairs;
    if ((rc = take(&p, sizeof(double) * ((size_t)npairs * 9 + nsys)))) return done(rc);
    S.rmax = (double*)p;
    S.xmax = S.rmax + npairs;
    S.bmax = S.xmax + npairs;
    S.dmax = S.bmax + npairs;
    S.dxmax = S.dmax + npairs;
    S.dprev = S.dxmax + npairs;
    S.relres = S.dprev + npairs;
    S.nbe = S.relres + npairs;
    S.anorm = S.nbe + npairs + npairs;  // one spare slot of npairs
    {
        // (failures release the buffers taken so far)
        cudaError_t e0 = cudaMemcpyAsync(d_order, hord.data(), sizeof(int32_t) * npairs, cudaMemcpyHostToDevice, s);
        if (!e0) e0 = cudaMemsetAsync(S.status, 0, sizeof(int32_t) * npairs * 3, s);
        if (!e0) e0 = cudaMemsetAsync(S.rmax, 0, sizeof(double) * ((size_t)npairs * 9 + nsys), s);
        if (e0) return done(cuda_error(e0, "batch state", __FILE__, __LINE__));
    }
    {
        ProfScope ps(BSPAI_K_OTHER, s);
        k_slice_seg_b<<<(unsigned)ceil_div(nsys, 256), 256, 0, s>>>(nsys, row_off, d_seg);
        note_launch();
        k_fill_d<<<(unsigned)ceil_div(npairs, 256), 256, 0, s>>>(npairs, S.dprev, INFINITY);
        note_launch();
        if (n > 0) {
            k_system_norms<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, A->sell.sptr, A->sell.col, A->val64, d_seg,
                                                                      S.anorm);
            note_launch();
            k_pair_bmax<<<(unsigned)ceil_div((int64_t)n * nrhs, 256), 256, 0, s>>>(n, nrhs, nsys, Bv, d_seg, S.bmax);
            note_launch();
        }
        {
            const cudaError_t e0 = cudaGetLastError();
            if (e0) return done(cuda_error(e0, "batch set-up kernels", __FILE__, __LINE__));
        }
        // x0 = M b in u_f for every right-hand side (Alg 3.1)
        if (!o.x0_given)
            for (int r = 0; r < nrhs; ++r)
                if ((rc = launch_apply_uf(M, Bv + (size_t)r * n, X + (size_t)r * n, s)))
                    return done(rc);
    }
    const BMDev Av = single_bucket_view(A->sell, u_p == BSPAI_FP64 ? (const void*)A->val64 : (const void*)A->val32,
                                        u_p);
    const BMDev Mv = BM->dev();
    // schedule: forced by the caller's thread, cached per batch shape, or tuned below
    const size_t ws_budget = (size_t)24 << 30;
    const int sms = num_sms();
    const int nmax32 = (int)ceil_div(nmax > 0 ? nmax : 1, 32) * 32;
    auto grid_for = [&](const Sched& c, int* grid) -> int {
        int occ = 0;
        int r2 = occupancy_blocks<T>(batch_kernel<T>(c.urows, c.msched), c.bd, sizeof(T) * (size_t)c.zcap, &occ);
        if (r2) return r2;
        if (occ < 1) return set_error(BSPAI_ERR_CUDA, "batched GMRES kernel does not fit on an SM");
        const size_t per = sizeof(T) * (size_t)ldv * (kmax + 2) + sizeof(double) * (size_t)ldv +
                           sizeof(double) * ((size_t)(kmax + 1) * kmax + 4 * (kmax + 2));
        int gmax = (int)(ws_budget / per);
        int gr = sms * occ;
        if (o.max_blocks > 0 && gr > o.max_blocks) gr = o.max_blocks;
        if (gr > gmax) gr = gmax;
        if (gr > npairs) gr = npairs;
        *grid = gr < 1 ? 1 : gr;
        return BSPAI_OK;
    };
    // the z-in-shared-memory limit of each (tile, CTA size), which also raises the
    // kernels' dynamic shared memory limit before any launch
    const int cand_bd[3] = {128, 256, 512};
    int zlim[2][2][3];  // [tile][bucket schedule][CTA size]: rows of z that fit
    for (int u = 0; u < 2; ++u)
        for (int m = 0; m < 2; ++m)
            for (int c = 0; c < 3; ++c)
                if ((rc = zcap_limit<T>(batch_kernel<T>(u ? MgsU<T>::hi : MgsU<T>::lo, m), cand_bd[c],
                                        &zlim[u][m][c])))
                    return done(rc);
    auto zfit = [&](const Sched& c) {
        const int u = c.urows == MgsU<T>::hi ? 1 : 0;
        for (int k = 0; k < 3; ++k)
            if (cand_bd[k] == c.bd) return zlim[u][c.msched ? 1 : 0][k];
        return 0;
    };
    // the candidate the tuner tries: every pair of the batch, if it fits
    auto zlimit = [&](const Sched& c) {
        const int z = zfit(c);
        return z < nmax32 ? z : nmax32;
    };
    Sched sch;
    sch.urows = MgsU<T>::lo;
    bool have = false;
    const TuneKey key{n, nsys, nrhs, ug, kmax};
    if (t_forced) {
        sch = t_force;
        if (sch.urows == 0) sch.urows = MgsU<T>::lo;
        if (sch.urows != MgsU<T>::lo && sch.urows != MgsU<T>::hi)
            return done(set_error(BSPAI_ERR_INVALID, "batch schedule: mgs_rows must be %d or %d for this u_g",
                                  MgsU<T>::lo, MgsU<T>::hi));
        if (sch.team > 0 && sizeof(T) != 4)
            return done(set_error(BSPAI_ERR_UNSUPPORTED, "batch schedule: team mode needs u_g = FP32"));
        if (sch.zcap < 0) sch.zcap = zlimit(sch);  // as many rows as fit
        if (sch.zcap > zfit(sch))
            return done(set_error(BSPAI_ERR_INVALID,
                                  "batch schedule: z_shared_rows %d exceeds the %d rows that fit in shared memory "
                                  "at this CTA size and tile",
                                  sch.zcap, zfit(sch)));
        if (sch.zcap > nmax32) sch.zcap = nmax32;  // no pair is larger: the same schedule
        have = true;
    } else {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            sch = it->second;
            have = true;
        }
    }
    // workspace for the largest grid among the candidates
    int gmax_all = 0;
    for (int u = 0; u < 2; ++u)
        for (int m = 0; m < 2; ++m)
            for (int c = 0; c < 3; ++c)
                for (int zs = 0; zs < 2; ++zs) {
                    Sched cs;
                    cs.bd = cand_bd[c];
                    cs.urows = u ? MgsU<T>::hi : MgsU<T>::lo;
                    cs.msched = m;
                    cs.zcap = zs ? (zlim[u][m][c] < nmax32 ? zlim[u][m][c] : nmax32) : 0;
                    int gr;
                    if ((rc = grid_for(cs, &gr))) return done(rc);
                    gmax_all = gr > gmax_all ? gr : gmax_all;
                }
    if (have) {
        int gr;
        if ((rc = grid_for(sch, &gr))) return done(rc);
        gmax_all = gr > gmax_all ? gr : gmax_all;
    }
    T *Vws = nullptr, *Wws = nullptr;
    double *Yws = nullptr, *Hws = nullptr, *Sws = nullptr;
    if ((rc = take((void**)&Vws, sizeof(T) * (size_t)gmax_all * ldv * (kmax + 1)))) return done(rc);
    if ((rc = take((void**)&Wws, sizeof(T) * (size_t)gmax_all * ldv))) return done(rc);
    if ((rc = take((void**)&Yws, sizeof(double) * (size_t)gmax_all * ldv))) return done(rc);
    if ((rc = take((void**)&Hws, sizeof(double) * (size_t)gmax_all * (kmax + 1) * kmax))) return done(rc);
    if ((rc = take((void**)&Sws, sizeof(double) * (size_t)gmax_all * 4 * (kmax + 2)))) return done(rc);
    unsigned long long* d_work = nullptr;  // algorithmic work counters of the GMRES launches
    if ((rc = take((void**)&d_work, 2 * sizeof(unsigned long long)))) return done(rc);
    auto launch_gmres = [&](const Sched& c, int grid, const double* Rin, double* Xout, int kcap, double tcap,
                            PairState& St, cudaStream_t st, int np) {
        batch_kernel<T>(c.urows, c.msched)<<<grid, c.bd, sizeof(T) * (size_t)c.zcap, st>>>(
            Av, Mv, row_off, nsys, n, d_order, np, d_queue, St.status, Rin, Xout, Vws, Wws, Yws, ldv, Hws, Sws,
            kcap, tcap, c.zcap, St.iters, St.steps, St.relres, St.dmax, St.dxmax, d_work);
        note_launch();
        return cudaGetLastError();
    };
    // ---- team mode (u_g = fp32): the size-sorted pairs split into runs of equal team
    // size G = ceil(n_s / team_rows); all runs at once in one cooperative launch (several
    // launches only if the runs' smallest teams do not fit the GPU together), each run a
    // group of CTAs in proportion to its MGS work, estimated as the sum of n_s^2 (GMRES
    // steps grow with the grid size, and an MGS pass reads n_s rows)
    const int team_cands[2] = {kTeamP * 2 * kTeamBD, kTeamP * kTeamBD};  // 8,192 and 4,096 rows
    const size_t team_smem = sizeof(float) * (size_t)(kmax + 1);
    int occ_team = 0;
    // every pair's rows must fit its team: at most kTeamMaxG CTAs of kTeamP * 2 * kTeamBD rows
    const bool team_fits = nmax <= kTeamMaxG * kTeamP * 2 * kTeamBD;
    if (t_forced && sch.team > 0 && !team_fits)
        return done(set_error(BSPAI_ERR_UNSUPPORTED, "batch schedule: team mode holds systems of at most %d rows",
                              kTeamMaxG * kTeamP * 2 * kTeamBD));
    if constexpr (sizeof(T) == 4) if (team_fits) {
        cudaError_t e0 = cudaFuncSetAttribute(k_gmres_team<kTeamP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)team_smem);
        if (!e0) e0 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_team, k_gmres_team<kTeamP>, kTeamBD,
                                                                    team_smem);
        if (e0) return done(cuda_error(e0, "team kernel occupancy", __FILE__, __LINE__));
    }
    int team_slots = sms * (occ_team > 0 ? occ_team : 1);  // co-resident CTAs of a team launch
    if (o.max_blocks > 0 && team_slots > o.max_blocks) team_slots = o.max_blocks;
    auto sys_rows = [&](int pair) { return hoff[pair % nsys + 1] - hoff[pair % nsys]; };
    struct TeamLaunch {
        std::vector<TeamGroup> g;
        int grid = 0;
    };
    // the launches (normally one) of team mode over the first np pairs; workspace offsets
    // for kcap Arnoldi steps
    auto plan_teams = [&](int tr, int np, int kcap, std::vector<TeamLaunch>& out) {
        out.clear();
        struct Run {
            int G, begin, count;
            int64_t ldv;
            double w;
        };
        std::vector<Run> runs;
        auto gof = [&](int pr) {
            const int gg = (sys_rows(pr) + tr - 1) / tr;
            return gg < 1 ? 1 : (gg > kTeamMaxG ? kTeamMaxG : gg);
        };
        for (int b = 0; b < np;) {
            const int G = gof(hord[b]);
            int e = b, nsmax = 0;
            double w = 0.0;
            while (e < np && gof(hord[e]) == G) {
                const double ns = (double)sys_rows(hord[e]);
                nsmax = (int)ns > nsmax ? (int)ns : nsmax;
                w += ns * ns;
                ++e;
            }
            runs.push_back(Run{G, b, e - b, ceil_div(nsmax > 0 ? nsmax : 1, 64) * 64, w > 0.0 ? w : 1.0});
            b = e;
        }
        // pack the runs into launches whose one-team-each minimum fits the slots
        size_t r0 = 0;
        while (r0 < runs.size()) {
            size_t r1 = r0;
            int need = 0;
            while (r1 < runs.size() && r1 - r0 < (size_t)kTeamMaxGroups && need + runs[r1].G <= team_slots)
                need += runs[r1++].G;
            if (r1 == r0) ++r1;  // a single run wider than the slots cannot occur (G <= 32 < slots)
            double wsum = 0.0;
            for (size_t r = r0; r < r1; ++r) wsum += runs[r].w;
            std::vector<int> nt(r1 - r0);
            int used = 0;
            for (size_t r = r0; r < r1; ++r) {
                int t = (int)((runs[r].w / wsum) * team_slots / runs[r].G);
                t = t < 1 ? 1 : t;
                t = t > runs[r].count ? runs[r].count : t;
                nt[r - r0] = t;
                used += t * runs[r].G;
            }
            while (used > team_slots) {  // too many: take teams from the most generously served run
                size_t best = r1;
                double bv = -1.0;
                for (size_t r = r0; r < r1; ++r)
                    if (nt[r - r0] > 1 && nt[r - r0] * runs[r].G / runs[r].w > bv) {
                        bv = nt[r - r0] * runs[r].G / runs[r].w;
                        best = r;
                    }
                if (best == r1) break;
                --nt[best - r0];
                used -= runs[best].G;
            }
            while (true) {  // CTAs left over: a team more for the most poorly served run that fits
                size_t best = r1;
                double bv = 1e300;
                for (size_t r = r0; r < r1; ++r)
                    if (nt[r - r0] < runs[r].count && used + runs[r].G <= team_slots &&
                        nt[r - r0] * runs[r].G / runs[r].w < bv) {
                        bv = nt[r - r0] * runs[r].G / runs[r].w;
                        best = r;
                    }
                if (best == r1) break;
                ++nt[best - r0];
                used += runs[best].G;
            }
            TeamLaunch L;
            int64_t voff = 0, woff = 0, hoffs = 0, soff = 0, toff = 0;
            for (size_t r = r0; r < r1; ++r) {
                TeamGroup gg;
                gg.G = runs[r].G;
                gg.begin = runs[r].begin;
                gg.count = runs[r].count;
                gg.cta0 = L.grid;
                gg.nteams = nt[r - r0];
                gg.ldv = runs[r].ldv;
                gg.voff = voff;
                gg.woff = woff;
                gg.hoff = hoffs;
                gg.soff = soff;
                gg.toff = toff;
                voff += (int64_t)gg.nteams * gg.ldv * (kcap + 1);
                woff += (int64_t)gg.nteams * gg.ldv;
                hoffs += (int64_t)gg.nteams * (kcap + 1) * kcap;
                soff += (int64_t)gg.nteams * 4 * (kcap + 2);
                toff += (int64_t)gg.nteams * 4 * gg.G;
                L.grid += gg.nteams * gg.G;
                L.g.push_back(gg);
            }
            out.push_back(L);
            r0 = r1;
        }
    };
    // workspace: the largest launch of every candidate, over the whole batch and the
    // tuning sample
    int64_t tv = 0, tw = 0, th = 0, tsd = 0;
    int tgrid = 0;
    auto need_ws = [&](int tr, int np) {
        std::vector<TeamLaunch> ls;
        plan_teams(tr, np, kmax, ls);
        for (const TeamLaunch& L : ls) {
            int64_t v = 0, w = 0, h = 0, sd = 0;
            for (const TeamGroup& gg : L.g) {
                v += (int64_t)gg.nteams * gg.ldv * (kmax + 1);
                w += (int64_t)gg.nteams * gg.ldv;
                h += (int64_t)gg.nteams * (kmax + 1) * kmax;
                sd += (int64_t)gg.nteams * 4 * (kmax + 2);
            }
            tv = v > tv ? v : tv;
            tw = w > tw ? w : tw;
            th = h > th ? h : th;
            tsd = sd > tsd ? sd : tsd;
            tgrid = L.grid > tgrid ? L.grid : tgrid;
        }
    };
    const int np_sample = npairs < 4 * sms ? npairs : 4 * sms;  // the tuner's sample (below)
    if (occ_team > 0) {
        for (int tr : team_cands) {
            need_ws(tr, npairs);
            need_ws(tr, np_sample);
        }
        if (t_forced && sch.team > 0) need_ws(sch.team, npairs);
    }
    float *TV = nullptr, *TW = nullptr, *TZ = nullptr;
    double *TH = nullptr, *TS = nullptr;
    unsigned long long* Ttags = nullptr;
    GridBar* Tbar = nullptr;
    int* d_tq = nullptr;  // one queue per group
    if (occ_team > 0) {
        if ((rc = take((void**)&TV, sizeof(float) * (size_t)tv))) return done(rc);
        if ((rc = take((void**)&TW, sizeof(float) * (size_t)tw))) return done(rc);
        if ((rc = take((void**)&TZ, sizeof(float) * (size_t)tw))) return done(rc);
        if ((rc = take((void**)&TH, sizeof(double) * (size_t)th))) return done(rc);
        if ((rc = take((void**)&TS, sizeof(double) * (size_t)tsd))) return done(rc);
        if ((rc = take((void**)&Ttags, sizeof(unsigned long long) * 4 * (size_t)tgrid))) return done(rc);
        if ((rc = take((void**)&Tbar, sizeof(GridBar)))) return done(rc);
        if ((rc = take((void**)&d_tq, sizeof(int) * kTeamMaxGroups))) return done(rc);
        cudaError_t e0 = cudaMemsetAsync(Tbar, 0, sizeof(GridBar), s);
        if (e0) return done(cuda_error(e0, "memset", __FILE__, __LINE__));
    }
    const unsigned long long team_tmo =
        (unsigned long long)((o.barrier_timeout_s > 0 ? o.barrier_timeout_s : 2.0) * 1e9);
    // team mode's launches over the first np pairs of the order
    auto launch_team = [&](int tr, int np, const double* Rin, double* Xout, int kcap, double tcap, PairState& St,
                           cudaStream_t st) -> cudaError_t {
        std::vector<TeamLaunch> ls;
        plan_teams(tr, np, kcap, ls);
        cudaError_t e = cudaSuccess;
        for (size_t i = 0; !e && i < ls.size(); ++i) {
            e = cudaMemsetAsync(d_tq, 0, sizeof(int) * kTeamMaxGroups, st);
            if (!e) e = cudaMemsetAsync(Ttags, 0, sizeof(unsigned long long) * 4 * (size_t)ls[i].grid, st);
            if (e) break;
            TeamArgs ta;
            ta.Av = Av;
            ta.Mv = Mv;
            ta.row_off = row_off;
            ta.nsys = nsys;
            ta.n = n;
            ta.order = d_order;
            ta.queue = d_tq;
            ta.status = St.status;
            ta.R = Rin;
            ta.X = Xout;
            ta.V = TV;
            ta.W = TW;
            ta.Z = TZ;
            ta.H = TH;
            ta.S = TS;
            ta.kmax = kcap;
            ta.tau = tcap;
            ta.ngroups = (int)ls[i].g.size();
            for (size_t k2 = 0; k2 < ls[i].g.size(); ++k2) ta.grp[k2] = ls[i].g[k2];
            ta.tags = Ttags;
            ta.bar = Tbar;
            ta.tmo = team_tmo;
            ta.iters = St.iters;
            ta.steps = St.steps;
            ta.relres = St.relres;
            ta.dmax = St.dmax;
            ta.dxmax = St.dxmax;
            ta.work = d_work;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)ls[i].grid);
            cfg.blockDim = dim3(kTeamBD);
            cfg.dynamicSmemBytes = team_smem;
            cfg.stream = st;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeCooperative;  // the CTAs of a team wait on one another
            at[0].val.cooperative = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            e = cudaLaunchKernelEx(&cfg, k_gmres_team<kTeamP>, ta);
            note_launch();
        }
        return e;
    };
    int tuned = 0;
    float tune_ms = 0.0f;
    if (!have) {
        // autotune: a fixed sample -- the largest pairs, four per SM (the batch's time is
        // in its large systems: MGS work grows with n_s k^2), 32 Arnoldi steps each
        // (tau = 0) on the right-hand sides, into scratch -- for each candidate of a
        // staged search (CTA size, then the MGS tile, then z in shared memory, then the
        // bucket schedule), each stage keeping the fastest so far.  Timing every pair
        // for 8 steps instead weighted the small systems and early steps, and picked
        // 256-thread CTAs that ran the 512 x 8 batch 15 % slower than 512.
        const int np_tune = np_sample;
        const int k_tune = kmax < 32 ? kmax : 32;
        double* Xs = nullptr;
        void* ps2 = nullptr;
        if ((rc = take((void**)&Xs, sizeof(double) * (size_t)n * nrhs))) return done(rc);
        if ((rc = take(&ps2, sizeof(int32_t) * npairs * 2 + sizeof(double) * npairs * 3))) return done(rc);
        PairState T2 = S;
        T2.iters = (int32_t*)ps2;
        T2.steps = T2.iters + npairs;
        T2.relres = (double*)(T2.steps + npairs);
        T2.dmax = T2.relres + npairs;
        T2.dxmax = T2.dmax + npairs;
        // every failure below goes through done(), which releases the buffers taken
        // above; the events are destroyed on every way out of this block
        struct Events {
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            ~Events() {
                if (e0) cudaEventDestroy(e0);
                if (e1) cudaEventDestroy(e1);
            }
        } ev;
#define BSPAI_TUNE_TRY(expr)                                                         \
    do {                                                                             \
        cudaError_t _e = (expr);                                                     \
        if (_e != cudaSuccess) return done(cuda_error(_e, #expr, __FILE__, __LINE__)); \
    } while (0)
        BSPAI_TUNE_TRY(cudaEventCreate(&ev.e0));
        BSPAI_TUNE_TRY(cudaEventCreate(&ev.e1));
        std::vector<bspai_batch_schedule_t> tab_s;
        std::vector<float> tab_ms;
        float best = 1e30f;
        auto trial = [&](const Sched& c) -> int {
            int gr;
            int r2 = grid_for(c, &gr);
            if (r2) return r2;
            BSPAI_TUNE_TRY(cudaMemsetAsync(d_queue, 0, sizeof(int), s));
            BSPAI_TUNE_TRY(cudaMemsetAsync(Xs, 0, sizeof(double) * (size_t)n * nrhs, s));
            BSPAI_TUNE_TRY(cudaEventRecord(ev.e0, s));
            if (c.team > 0) BSPAI_TUNE_TRY(launch_team(c.team, np_tune, Bv, Xs, k_tune, 0.0, T2, s));
            else BSPAI_TUNE_TRY(launch_gmres(c, gr, Bv, Xs, k_tune, 0.0, T2, s, np_tune));
            BSPAI_TUNE_TRY(cudaEventRecord(ev.e1, s));
            BSPAI_TUNE_TRY(cudaEventSynchronize(ev.e1));
            float ms = 0;
            BSPAI_TUNE_TRY(cudaEventElapsedTime(&ms, ev.e0, ev.e1));
            tab_s.push_back(bspai_batch_schedule_t{c.bd, c.urows, c.zcap, c.msched, c.team});
            tab_ms.push_back(ms);
            tune_ms += ms;
            ++tuned;
            if (ms < best) {
                best = ms;
                sch = c;
            }
            return BSPAI_OK;
        };
        for (int c = 0; c < 3; ++c) {
            Sched cs;
            cs.bd = cand_bd[c];
            cs.urows = MgsU<T>::lo;
            if ((rc = trial(cs))) return done(rc);
        }
        {
            Sched cs = sch;
            cs.urows = MgsU<T>::hi;
            if ((rc = trial(cs))) return done(rc);
        }
        if (zlimit(sch) >= 32) {
            Sched cs = sch;
            cs.zcap = zlimit(sch);
            if ((rc = trial(cs))) return done(rc);
        }
        {
            Sched cs = sch;
            cs.msched = 1;
            if ((rc = trial(cs))) return done(rc);
        }
        // team mode, when every pair takes the same team size: the sample (the largest
        // pairs) then stands for the batch.  On a batch of many sizes it does not: its
        // small pairs run their products from L2 (a team's CTAs write the vectors they
        // gather) on teams sized for them or, at the end, on larger ones; on the 512 x 32
        // batch the sample favoured team mode by 9 % and the whole batch ran 13 % slower
        if (occ_team > 0)
            for (int tr : team_cands) {
                std::vector<TeamLaunch> ls;
                plan_teams(tr, npairs, kmax, ls);
                if (ls.size() != 1 || ls[0].g.size() != 1) continue;
                Sched cs;
                cs.bd = kTeamBD;
                cs.urows = MgsU<T>::lo;
                cs.team = tr;
                if ((rc = trial(cs))) return done(rc);
            }
        // a team exchange that ran out of time during tuning is an error like any other
        {
            int terr = 0;
            if (Tbar) BSPAI_TUNE_TRY(cudaMemcpy(&terr, &Tbar->err, sizeof(int), cudaMemcpyDeviceToHost));
            if (terr) return done(set_error(BSPAI_TIMEOUT, "batched solve: a team exchange exceeded its time limit"));
        }
#undef BSPAI_TUNE_TRY
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = sch;
        g_table_s = tab_s;
        g_table_ms = tab_ms;
    }
    const int bd = sch.bd;
    int grid = 0;
    if ((rc = grid_for(sch, &grid))) return done(rc);
    {
        cudaError_t e0 = cudaMemsetAsync(d_work, 0, 2 * sizeof(unsigned long long), s);
        if (e0) return done(cuda_error(e0, "memset", __FILE__, __LINE__));
    }
    // one refinement step: residuals, tests, the persistent GMRES launch, tests
    auto step = [&](cudaStream_t st) -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(S.rmax, 0, sizeof(double) * npairs * 2, st);  // rmax, xmax
        if (!e) e = cudaMemsetAsync(d_queue, 0, sizeof(int) * 2, st);                // queue, active
        if (e) return e;
        if (launch_residual_batch(A, nrhs, X, Bv, R, d_seg, nsys, S.rmax, S.xmax, st)) return cudaErrorUnknown;
        k_batch_flags<<<(unsigned)ceil_div(npairs, 256), 256, 0, st>>>(npairs, nsys, S, ustop, d_active);
        note_launch();
        {
            ProfScope ps(BSPAI_K_MGS, st);
            if (sch.team > 0) {
                if ((e = launch_team(sch.team, npairs, R, X, kmax, tau, S, st))) return e;
            } else if ((e = launch_gmres(sch, grid, R, X, kmax, tau, S, st, npairs))) {
                return e;
            }
        }
        k_batch_after<<<(unsigned)ceil_div(npairs, 256), 256, 0, st>>>(npairs, S, ustop, stag);
        note_launch();
        return cudaGetLastError();
    };
    static thread_local int* t_active = nullptr;  // [0]: pairs still active, [1]: a team exchange timed out
    if (!t_active) {
        cudaError_t e = cudaMallocHost(&t_active, 2 * sizeof(int));
        if (e != cudaSuccess) {
            t_active = nullptr;
            return done(cuda_error(e, "cudaMallocHost(active flag)", __FILE__, __LINE__));
        }
    }
    // Every refinement step issues the same five operations on the same buffers, so the
    // sequence is captured once into a CUDA graph and replayed.  Capture runs on a private
    // stream (the legacy default stream cannot be captured); replays go to the caller's
    // stream.  With kernel-class profiling on, the step is launched directly so that its
    // events land on the caller's stream.
    struct GraphGuard {
        cudaGraphExec_t e = nullptr;
        ~GraphGuard() {
            if (e) cudaGraphExecDestroy(e);
        }
    } gexec;
    long long graph_kernels = 0;
    if (!prof_enabled()) {
        cudaStream_t cs = nullptr;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (!e) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (!e) {
            count_launches(false);  // the replays are counted, not the capture
            cudaError_t e2 = step(cs);
            count_launches(true);
            e = cudaStreamEndCapture(cs, &g);
            if (!e) e = e2;
        }
        if (!e) e = cudaGraphInstantiate(&gexec.e, g, 0);
        if (!e) {
            size_t nn = 0;
            e = cudaGraphGetNodes(g, nullptr, &nn);
            std::vector<cudaGraphNode_t> nodes(nn);
            if (!e && nn) e = cudaGraphGetNodes(g, nodes.data(), &nn);
            for (size_t i = 0; !e && i < nn; ++i) {
                cudaGraphNodeType t;
                e = cudaGraphNodeGetType(nodes[i], &t);
                graph_kernels += !e && t == cudaGraphNodeTypeKernel;
            }
        }
        if (g) cudaGraphDestroy(g);
        if (cs) cudaStreamDestroy(cs);
        if (e) {
            // a step that cannot be captured (e.g. its cooperative team launches) runs directly
            (void)cudaGetLastError();
            if (gexec.e) cudaGraphExecDestroy(gexec.e);
            gexec.e = nullptr;
            graph_kernels = 0;
        }
    }
    int ir = 0, launched = 0;
    for (; ir < imax; ++ir) {
        ++launched;
        cudaError_t e;
        if (gexec.e) {
            e = cudaGraphLaunch(gexec.e, s);
            for (long long k = 0; k < graph_kernels; ++k) note_launch();
        } else {
            e = step(s);
        }
        t_active[1] = 0;
        if (!e) e = cudaMemcpyAsync(t_active, d_active, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (!e && Tbar) e = cudaMemcpyAsync(t_active + 1, &Tbar->err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) return done(cuda_error(e, "batched refinement step", __FILE__, __LINE__));
        if (t_active[1]) return done(set_error(BSPAI_TIMEOUT, "batched solve: a team exchange exceeded its time limit"));
        if (t_active[0] == 0) break;
    }
    // results (a failure still releases the buffers through done())
#define BSPAI_RES_TRY(expr)                                                          \
    do {                                                                             \
        cudaError_t _e = (expr);                                                     \
        if (_e != cudaSuccess) return done(cuda_error(_e, #expr, __FILE__, __LINE__)); \
    } while (0)
    std::vector<int32_t> hst(npairs), hit(npairs), hsteps(npairs);
    std::vector<double> hnbe(npairs);
    BSPAI_RES_TRY(cudaMemcpyAsync(hst.data(), S.status, sizeof(int32_t) * npairs, cudaMemcpyDeviceToHost, s));
    BSPAI_RES_TRY(cudaMemcpyAsync(hit.data(), S.iters, sizeof(int32_t) * npairs, cudaMemcpyDeviceToHost, s));
    BSPAI_RES_TRY(cudaMemcpyAsync(hsteps.data(), S.steps, sizeof(int32_t) * npairs, cudaMemcpyDeviceToHost, s));
    BSPAI_RES_TRY(cudaMemcpyAsync(hnbe.data(), S.nbe, sizeof(double) * npairs, cudaMemcpyDeviceToHost, s));
    if (pair_status) BSPAI_RES_TRY(cudaMemcpyAsync(pair_status, S.status, sizeof(int32_t) * npairs, cudaMemcpyDeviceToDevice, s));
    if (pair_iters) BSPAI_RES_TRY(cudaMemcpyAsync(pair_iters, S.iters, sizeof(int32_t) * npairs, cudaMemcpyDeviceToDevice, s));
    unsigned long long hwork[2] = {0, 0};
    BSPAI_RES_TRY(cudaMemcpyAsync(hwork, d_work, sizeof hwork, cudaMemcpyDeviceToHost, s));
    BSPAI_RES_TRY(cudaStreamSynchronize(s));
#undef BSPAI_RES_TRY
    int conv = 0, nonfin = 0, maxit = 0, maxsteps = 0;
    int64_t tot = 0;
    for (int q = 0; q < npairs; ++q) {
        conv += hst[q] > 0;
        nonfin += hst[q] < 0;
        tot += hit[q];
        maxit = hit[q] > maxit ? hit[q] : maxit;
        maxsteps = hsteps[q] > maxsteps ? hsteps[q] : maxsteps;
    }
    if (info) {
        info->pairs = npairs;
        info->converged = conv;
        info->nonfinite = nonfin;
        info->ir_launches = launched;
        info->max_ir_steps = maxsteps;
        info->total_iters = tot;
        info->max_iters = maxit;
        info->block_threads = bd;
        info->grid = grid;
        info->kmax = kmax;
        info->mgs_rows = sch.urows;
        info->z_shared_rows = sch.zcap;
        info->m_schedule = sch.msched;
        info->team_rows = sch.team;
        // algorithmic bytes of the GMRES launches: each MGS pass reads one basis vector's
        // rows once (the last pass none, and v_{j+1} is written: j + 2 row-vectors per
        // step); each step's A v and M w read A (values in u_p, int32 columns) and the
        // bucketed M (stored values, int32 columns, e4m3 column scales) of the pair's
        // rows at the batch's average entries per row, and gather / write four vectors
        const double es = (double)sizeof(T);
        const double upb = u_p == BSPAI_FP64 ? 8.0 : 4.0;
        double mb = 0.0;
        for (int k = 0; k < BM->q; ++k) {
            const int f = BM->precs[k];
            const double vb = f == BSPAI_FP64 ? 8 : f == BSPAI_FP32 ? 4 : (f == BSPAI_FP16 || f == BSPAI_BF16) ? 2
                                                                      : f == BSPAI_E4M3 ? 1 : -1;
            if (vb > 0) mb += (double)BM->nnz_k[k] * (vb + 4.0);
            if (f == BSPAI_E4M3) mb += 4.0 * n;
        }
        const double per_row = n > 0 ? ((double)A->nnz * (upb + 4.0) + mb) / n + 4.0 * es : 0.0;
        info->gmres_bytes = (int64_t)((double)hwork[0] * es + (double)hwork[1] * per_row);
        info->tuned_candidates = tuned;
        info->tune_ms = tune_ms;
    }
    done(BSPAI_OK);
    if (nonfin) return set_error(BSPAI_NONFINITE, "batched solve: %d pairs hit a non-finite value", nonfin);
    if (conv < npairs)
        return set_error(BSPAI_NOT_CONVERGED, "batched solve: %d of %d pairs met no stopping test", npairs - conv,
                         npairs);
    return BSPAI_OK;
}

}  // namespace bspai

using namespace bspai;

extern "C" {

int bspai_batch_schedule_force(const bspai_batch_schedule_t* sched) {
    if (!sched) {
        t_forced = false;
        return BSPAI_OK;
    }
    if (sched->block_threads != 128 && sched->block_threads != 256 && sched->block_threads != 512)
        return set_error(BSPAI_ERR_INVALID, "bspai_batch_schedule_force: block_threads must be 128, 256 or 512");
    if (sched->m_schedule != 0 && sched->m_schedule != 1)
        return set_error(BSPAI_ERR_INVALID, "bspai_batch_schedule_force: m_schedule must be 0 or 1");
    if (sched->z_shared_rows < -1 || sched->mgs_rows < 0)
        return set_error(BSPAI_ERR_INVALID, "bspai_batch_schedule_force: negative field");
    if (sched->team_rows != 0 &&
        (sched->team_rows < 1024 || sched->team_rows > kTeamP * 2 * kTeamBD || sched->team_rows % 1024))
        return set_error(BSPAI_ERR_INVALID,
                         "bspai_batch_schedule_force: team_rows must be 0 or a multiple of 1024 up to %d",
                         kTeamP * 2 * kTeamBD);
    t_force.bd = sched->block_threads;
    t_force.urows = sched->mgs_rows;
    t_force.zcap = sched->z_shared_rows;
    t_force.msched = sched->m_schedule;
    t_force.team = sched->team_rows;
    t_forced = true;
    return BSPAI_OK;
}

int bspai_batch_tune_table(bspai_batch_schedule_t* sched, float* ms, int32_t cap, int32_t* count) {
    if (!count || cap < 0 || (cap > 0 && (!sched || !ms)))
        return set_error(BSPAI_ERR_INVALID, "bspai_batch_tune_table: bad arguments");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    *count = (int32_t)g_table_s.size();
    for (int32_t i = 0; i < cap && i < *count; ++i) {
        sched[i] = g_table_s[i];
        ms[i] = g_table_ms[i];
    }
    return BSPAI_OK;
}

int gmres_ir_solve_batched(bspai_A_h A, const int32_t* row_off, int32_t nsys, int32_t nrhs, const double* B,
                           bspai_BM_h BM, bspai_M_h M, bspai_prec_t u_g, bspai_prec_t u_p, double tol,
                           const bspai_opts_t* opts, double* X, bspai_stream_t st, bspai_batch_info_t* info,
                           int32_t* pair_status, int32_t* pair_iters) {
    cudaStream_t s = (cudaStream_t)st;
    if (!A || A->magic != kMagicA) return set_error(BSPAI_ERR_INVALID, "gmres_ir_solve_batched: bad A handle");
    if (!BM || BM->magic != kMagicBM) return set_error(BSPAI_ERR_INVALID, "gmres_ir_solve_batched: bad M handle");
    if (M && M->magic != kMagicM) return set_error(BSPAI_ERR_INVALID, "gmres_ir_solve_batched: bad M handle");
    if (nsys < 1 || nrhs < 1 || !row_off || !B || !X)
        return set_error(BSPAI_ERR_INVALID, "gmres_ir_solve_batched: bad batch description");
    if (BM->n != A->n || (M && M->n != A->n)) return set_error(BSPAI_ERR_INVALID, "gmres_ir_solve_batched: size mismatch");
    for (int k = 0; k < BM->q; ++k)
        if (BM->b[k].packed || BM->b[k].col16)
            return set_error(BSPAI_ERR_INVALID,
                             "gmres_ir_solve_batched: M must come from bspai_bucket_batched (its slot arrangement)");
    if ((A->n & 31) != 0) return set_error(BSPAI_ERR_INVALID, "gmres_ir_solve_batched: n must be a multiple of 32");
    if (u_g != BSPAI_FP32 && u_g != BSPAI_FP64) return set_error(BSPAI_ERR_UNSUPPORTED, "u_g must be FP32 or FP64");
    if (u_p != BSPAI_FP32 && u_p != BSPAI_FP64) return set_error(BSPAI_ERR_UNSUPPORTED, "u_p must be FP32 or FP64");
    bspai_opts_t o;
    bspai_opts_default(&o);
    if (opts) o = *opts;
    if (!o.x0_given && !M) return set_error(BSPAI_ERR_INVALID, "gmres_ir_solve_batched: need M for x0 = M b");
    if (info) memset(info, 0, sizeof *info);
    return u_g == BSPAI_FP64 ? batch_ir<double>(A, row_off, nsys, nrhs, B, BM, M, u_p, tol, o, X, s, info, pair_status,
                                                pair_iters)
                             : batch_ir<float>(A, row_off, nsys, nrhs, B, BM, M, u_p, tol, o, X, s, info, pair_status,
                                               pair_iters);
}

}  // extern "C"
