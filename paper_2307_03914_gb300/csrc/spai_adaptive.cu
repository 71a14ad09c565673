// spai_adaptive.cu -- adaptive sparse approximate inverse (Alg 2.1 with
// alpha > 0: Grote and Huckle's pattern growth) on the GPU.
//
// As for the fixed pattern, SPAI runs on B = A^T D (Section 4) and gives the
// left preconditioner M = M'^T D; column k of M' is row k of M and column j of
// B is row j of A times d_j.  Each column starts from the identity pattern
// J_k = {k} (Section 4) and repeats, at most alpha + 1 times:
//   I_k    = shadow of J_k (the union of the columns of rows J_k of A);
//   solve  min ||ebar - Abar mbar||_2 by Householder QR; sbar = Abar mbar - ebar;
//   stop   when ||sbar||_2 <= spai_eps, or after the last solve;
//   L_k    = I_k u {k};  Jt_k = (union over l in L_k of N_l) \ J_k, with
//            N_l = {j : b_lj != 0}, the rows of A with an entry in column l
//            (row l of A^T);
//   rho_j  = (||sbar||^2 - (sbar^T B(I_k, j))^2 / ||B e_j||^2)^(1/2), the
//            residual of the best update along e_j alone (Grote and Huckle's
//            univariate minimisation; sbar is zero outside I_k);
//   add    the up to beta indices of smallest rho_j (ties: smaller j) among
//          those with rho_j <= the mean of rho over Jt_k.
// A step whose new pattern would have a shadow of more than lmax rows is not
// taken (the column keeps its current solution and is marked capped): lmax
// bounds the shared memory of one column.
//
// One warp per column, every operation in u_f (fp32, or half through UfOps) as
// in the fixed-pattern kernel: the gathered rows of A (B's u_f values
// precomputed once), the
// shadow (bitonic sort + ballot compaction), Abar in shared memory, the
// Householder QR with warp-shuffle reductions (updated from pass to pass in
// fp32, see k_spai_adaptive), back substitution, sbar from the gathered
// entries; the candidates by one sweep over the rows of B in I_k
// into an open-addressing hash table that also accumulates sbar^T B(I_k, j)
// in exact fixed point (the u_f products summed exactly, then rounded once to
// u_f), rho per candidate from that sum and the precomputed
// ||B e_j||^2, the mean as a fixed-point sum, and beta rounds of a warp argmin
// over (rho, j) for the picks.  Every loop has a bound set by jmax, lmax or
// the host-computed buffer sizes.  Two launches (tiers) share the kernel; see
// k_spai_adaptive.
#include <climits>

#include "common.cuh"

namespace bspai {

int launch_row_absmax_inv(int n, const int32_t* row_ptr, const double* val, double* d, cudaStream_t s);

struct AdaptiveCounters {
    int n_conv;
    int n_rankdef;
    int n_capped;
    int max_cols;
    int max_rows;
    float max_resid;
    unsigned long long solves;
    int n_nonfinite;  // entries of M outside the range of u_f
};

// shared memory of one warp, 16-byte aligned pieces
struct AdaptiveLayout {
    size_t acc, J, Js, stp, rbeg, eoff, picks, mv, rdiag, tw, ecol, eq, eval, I, Is, Ip, cv, sv, tab, region, total;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// jmax, lmax: bounds on |J| and |I|; gmax: on the gathered entries of rows J;
// lp2: the shadow sort's length (a power of two >= gmax); H: the candidate
// hash table's size (a power of two; every candidate passes through it).  The
// table's storage (tab, acc) is also the scratch of the shadow sort and of the
// merge of new shadow rows, and holds the candidates and their rho while it is
// emptied: H >= lp2 and H >= lmax (the host sizes it so).  The region holds
// the factorised Abar from pass to pass.
__host__ __device__ inline AdaptiveLayout adaptive_layout(int jmax, int lmax, int gmax, int lp2, int H) {
    AdaptiveLayout L{};
    size_t o = 0;
    L.acc = o;   o += al16((size_t)H * 8);  // the candidates' fixed-point sbar^T B e_j
    L.J = o;     o += al16((size_t)jmax * 4);
    L.Js = o;    o += al16((size_t)jmax * 4);
    L.stp = o;   o += al16((size_t)jmax * 4);
    L.rbeg = o;  o += al16((size_t)jmax * 4);
    L.eoff = o;  o += al16((size_t)(jmax + 1) * 4);
    L.picks = o; o += al16((size_t)jmax * 4);
    L.mv = o;    o += al16((size_t)jmax * 4);
    L.rdiag = o; o += al16((size_t)jmax * 4);
    L.tw = o;    o += al16((size_t)jmax * 4);
    L.ecol = o;  o += al16((size_t)gmax * 4);
    L.eq = o;    o += al16((size_t)gmax * 4);
    L.eval = o;  o += al16((size_t)gmax * 4);
    L.I = o;     o += al16((size_t)lmax * 4);
    L.Is = o;    o += al16((size_t)lmax * 4);
    L.Ip = o;    o += al16((size_t)lmax * 4);
    L.cv = o;    o += al16((size_t)lmax * 4);
    L.sv = o;    o += al16((size_t)lmax * 4);
    L.tab = o;   o += al16((size_t)H * 4);
    L.region = o;  // Abar (column-major, leading dimension lmax)
    o += al16((size_t)lmax * jmax * 4);
    L.total = o;
    (void)lp2;
    return L;
}


// x * 2^40 as a 64-bit integer, truncated toward zero (|x| < 2^22), from the
// bits of x with integer operations only (64-bit float-integer conversions
// would use the narrow fp64 pipe)
__device__ __forceinline__ long long fix40(float x) {
    const unsigned u = __float_as_uint(x);
    const int e = (int)((u >> 23) & 0xFFu);
    if (e == 0) return 0;  // zero or subnormal: below 2^-126, nothing at 2^-40
    const long long m = (long long)((u & 0x7FFFFFu) | 0x800000u);
    const int sh = e - 110;  // x = m 2^(e - 150), times 2^40
    const long long r = sh >= 0 ? (m << sh) : (sh > -40 ? (m >> -sh) : 0);
    return (u >> 31) ? -r : r;
}

// v * 2^-40 as a float, from the two 32-bit halves of v
__device__ __forceinline__ float unfix40(long long v) {
    const float hi = (float)(int)(v >> 32);
    const float lo = (float)(unsigned)(v & 0xFFFFFFFFll);
    return __fmul_rn(__fadd_rn(__fmul_rn(hi, 4294967296.0f), lo), 9.094947017729282e-13f);
}

__device__ __forceinline__ int lb_i32(const int* a, int n, int v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool contains(const int* a, int n, int v) {
    const int p = lb_i32(a, n, v);
    return p < n && a[p] == v;
}

// bitonic sort of keys[0, LP), LP a power of two >= 2
__device__ __forceinline__ void warp_bitonic(int* keys, int LP, int lane) {
    for (int size = 2; size <= LP; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < (LP >> 1); t += 32) {
                const int i = ((t & ~(stride - 1)) << 1) | (t & (stride - 1));
                const int jj = i + stride;
                const bool asc = (i & size) == 0;
                const int a = keys[i], b = keys[jj];
                if ((a > b) == asc) {
                    keys[i] = b;
                    keys[jj] = a;
                }
            }
            __syncwarp();
        }
    }
}

__device__ __forceinline__ int pow2_at_least(int v) {
    int p = 32;
    while (p < v) p <<= 1;
    return p;
}

// Gather every entry of rows J[q0, q1) of A -- the columns added by a pass --
// after the L0 entries already gathered: its column, its value in B (a_jc d_j
// rounded to u_f, precomputed) and its q.  eoff[q] is the first entry of
// column q (eoff[q0] = L0 on entry).  Returns the new count (<= q1 * rowmax).
__device__ __forceinline__ int gather_new_rows(const int* J, int q0, int q1, int L0, const int32_t* __restrict__ arp,
                                               const int32_t* __restrict__ acol, const float* __restrict__ bval,
                                               int* rbeg, int* eoff, int* ecol, int* eq, float* eval, int lane) {
    for (int q = q0 + lane; q < q1; q += 32) {
        const int j = J[q];
        const int rb = arp[j];
        rbeg[q] = rb;
        eoff[q + 1] = arp[j + 1] - rb;  // lengths first, offsets below
    }
    __syncwarp();
    if (lane == 0) {
        eoff[q0] = L0;
        for (int q = q0; q < q1; ++q) eoff[q + 1] += eoff[q];
    }
    __syncwarp();
    const int L = eoff[q1];
    for (int t = L0 + lane; t < L; t += 32) {
        int lo = q0, hi = q1;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (eoff[mid] <= t) lo = mid;
            else hi = mid;
        }
        const int e = rbeg[lo] + (t - eoff[lo]);
        ecol[t] = acol[e];
        eval[t] = bval[e];
        eq[t] = lo;
    }
    __syncwarp();
    return L;
}

// The distinct columns among ecol[L0, L) that are not rows of the shadow yet
// (Is[0, nI), sorted), ascending, into out (at most room written); returns
// their number (which may exceed room).  keys: LP >= L - L0 ints of scratch,
// left holding -1.
__device__ __forceinline__ int new_shadow_rows(const int* ecol, int L0, int L, const int* Is, int nI, int* keys,
                                               int* out, int room, int lane) {
    const int cnt = L - L0;
    const int LP = pow2_at_least(cnt > 2 ? cnt : 2);
    for (int t = lane; t < LP; t += 32) keys[t] = t < cnt ? ecol[L0 + t] : INT_MAX;
    __syncwarp();
    warp_bitonic(keys, LP, lane);
    int nn = 0;
    for (int b0 = 0; b0 < cnt; b0 += 32) {
        const int t = b0 + lane;
        const int v = t < cnt ? keys[t] : INT_MAX;
        const int prev = (t > 0 && t < cnt) ? keys[t - 1] : -1;
        const bool flag = t < cnt && v != prev && !contains(Is, nI, v);
        const unsigned m = __ballot_sync(0xffffffffu, flag);
        const int pos = nn + __popc(m & ((1u << lane) - 1u));
        if (flag && pos < room) out[pos] = v;
        nn += __popc(m);
    }
    __syncwarp();
    for (int t = lane; t < LP; t += 32) keys[t] = -1;
    __syncwarp();
    return nn;
}

// Two tiers share this kernel.  The first runs every column with a small
// per-warp footprint (jmax, lmax below the full bounds, so more warps fit on
// an SM); a column whose pattern or shadow outgrows it -- without reaching the
// caller's cap_rows -- is appended to redo_list and left unwritten.  The second
// tier (redo_list == nullptr) reruns exactly those columns (cols) from the
// start with the full bounds.  Both run the same steps in the same order, so
// a column's result does not depend on the tier that finished it.
//
// QR updating (the remark after Alg 2.1, Grote and Huckle's eqs. 14-15): the
// Householder factorisation of Abar = B(I, J) is kept from pass to pass.  The
// rows of Abar stay in the order they joined the shadow (Is/Ip: the sorted
// row ids and their Abar rows, for lookups), the columns in the order they
// joined J.  A pass that adds columns Jt and rows It needs no new row in the
// old columns (B(It, J) = 0: It lies outside the old shadow), so Abar grows to
// [[Abar, B(I, Jt)], [0, B(It, Jt)]]: the old reflectors (zero on the new
// rows) are applied to the new columns, the new columns are factored below
// the old ones, and Q^T ebar keeps its old entries (ebar's new rows are zero,
// but for k).  The least-squares solution is that of a fresh factorisation up
// to rounding.
template <bool HALF>
__global__ void __launch_bounds__(256, 3) k_spai_adaptive(
    int n, int ncols, const int32_t* __restrict__ cols, const int32_t* __restrict__ arp,
    const int32_t* __restrict__ acol, const float* __restrict__ bval, const float* __restrict__ bnorm2,
    const double* __restrict__ d, const int32_t* __restrict__ trp, const int32_t* __restrict__ tcol,
    const float* __restrict__ tval, float spai_eps, float u_f, int alpha, int beta,
    int jmax, int lmax, int gmax, int lp2, int H, int cap_rows, int32_t* __restrict__ redo_list,
    int* __restrict__ redo_count,
    int32_t* __restrict__ Jo, float* __restrict__ Mo, int8_t* __restrict__ So, int32_t* __restrict__ nJo,
    float* __restrict__ resid, int32_t* __restrict__ cinfo, AdaptiveCounters* __restrict__ cnt) {
    using F = UfOps<HALF>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t idx = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (idx >= ncols) return;
    const int64_t k = cols ? (int64_t)cols[idx] : idx;
    const AdaptiveLayout LY = adaptive_layout(jmax, lmax, gmax, lp2, H);
    unsigned char* base = smem + LY.total * wib;
    long long* acc = reinterpret_cast<long long*>(base + LY.acc);
    int* J = reinterpret_cast<int*>(base + LY.J);    // in the order the columns joined
    int* Js = reinterpret_cast<int*>(base + LY.Js);  // the same, ascending (membership tests)
    int* stp = reinterpret_cast<int*>(base + LY.stp);
    int* rbeg = reinterpret_cast<int*>(base + LY.rbeg);
    int* eoff = reinterpret_cast<int*>(base + LY.eoff);
    int* picks = reinterpret_cast<int*>(base + LY.picks);
    float* mv = reinterpret_cast<float*>(base + LY.mv);
    float* rdiag = reinterpret_cast<float*>(base + LY.rdiag);
    float* tw = reinterpret_cast<float*>(base + LY.tw);  // 2 / v^T v of each reflector
    int* ecol = reinterpret_cast<int*>(base + LY.ecol);
    int* eq = reinterpret_cast<int*>(base + LY.eq);
    float* eval = reinterpret_cast<float*>(base + LY.eval);
    int* I = reinterpret_cast<int*>(base + LY.I);    // row id at each Abar row
    int* Is = reinterpret_cast<int*>(base + LY.Is);  // row ids ascending
    int* Ip = reinterpret_cast<int*>(base + LY.Ip);  // ... and their Abar rows
    float* cv = reinterpret_cast<float*>(base + LY.cv);
    float* sv = reinterpret_cast<float*>(base + LY.sv);
    int* tab = reinterpret_cast<int*>(base + LY.tab);
    float* Ab = reinterpret_cast<float*>(base + LY.region);  // column-major, leading dimension lmax
    // candidates and their rho reuse the hash table's storage while it is emptied
    int* keys = tab;
    float* rho = reinterpret_cast<float*>(acc);
    for (int t = lane; t < H; t += 32) {  // empty; every pass leaves it empty again
        tab[t] = -1;
        acc[t] = 0;
    }
    if (lane == 0) {
        J[0] = (int)k;
        Js[0] = (int)k;
        stp[0] = 0;
    }
    __syncwarp();
    int nJ = 1, nJ_old = 0;  // columns in J; columns already factored
    int L = 0, nI = 0;       // entries gathered; rows of Abar
    int max_rows = 0;
    float res_norm = 1.0f, r2sum = 1.0f, fro2 = 0.0f;
    bool rankdef = false, conv = false, capped = false, redo = false;
    int solves = 0;

    for (int step = 0; step <= alpha; ++step) {
        // ---- the new columns' rows of A, the shadow rows they add (checked against lmax
        // before anything of the current factorisation changes).  In u_f = half every
        // pass starts afresh instead, with Abar's rows in ascending order: half rounding
        // is coarse enough that another operation order (the updated factors' or the
        // rows' order of arrival) moves many near-tied picks against the fp64 scoring.
        const int q0 = HALF ? 0 : nJ_old;  // first column gathered (and factored) in this pass
        const int Lg = HALF ? 0 : L;       // its first entry
        const int Ln = gather_new_rows(J, q0, nJ, Lg, arp, acol, bval, rbeg, eoff, ecol, eq, eval, lane);
        // half: the whole shadow, ascending, into I (new: its rows beyond the old ones)
        const int nnew = HALF ? new_shadow_rows(ecol, 0, Ln, Is, 0, keys, I, lmax, lane) - nI
                              : new_shadow_rows(ecol, Lg, Ln, Is, nI, keys, I + nI, lmax - nI, lane);
        if (nI + nnew > lmax) {  // never on the first pass: rowmax <= lmax (host check)
            if (redo_list && nI + nnew <= cap_rows) redo = true;
            else capped = true;
            // the columns of this pass are not taken (in half they were merged into J:
            // they are the ones added for this step)
            if (HALF && lane == 0) {
                int w = 0;
                for (int q = 0; q < nJ; ++q)
                    if (stp[q] != step) {
                        J[w] = J[q];
                        stp[w] = stp[q];
                        ++w;
                    }
            }
            __syncwarp();
            nJ = nJ_old;
            break;
        }
        const int nIn = nI + nnew;
        if (HALF) {  // Abar's rows ascending: I is the sorted shadow
            for (int u = lane; u < nIn; u += 32) {
                Is[u] = I[u];
                Ip[u] = u;
            }
            __syncwarp();
        } else {
            // merge the new rows (I[nI, nIn), ascending) into Is / Ip, through keys and acc
            int* mIs = keys;
            int* mIp = reinterpret_cast<int*>(acc);
            for (int u = lane; u < nI; u += 32) {
                const int pos = u + lb_i32(I + nI, nnew, Is[u]);
                mIs[pos] = Is[u];
                mIp[pos] = Ip[u];
            }
            for (int m = lane; m < nnew; m += 32) {
                const int pos = m + lb_i32(Is, nI, I[nI + m]);
                mIs[pos] = I[nI + m];
                mIp[pos] = nI + m;
            }
            __syncwarp();
            for (int u = lane; u < nIn; u += 32) {
                Is[u] = mIs[u];
                Ip[u] = mIp[u];
            }
            __syncwarp();  // (mIp lives in acc: every entry is read before any is cleared)
            for (int u = lane; u < nIn; u += 32) {
                mIs[u] = -1;
                acc[u] = 0;
            }
            __syncwarp();
        }
        // the new entries' rows in Abar
        for (int t = Lg + lane; t < Ln; t += 32) ecol[t] = Ip[lb_i32(Is, nIn, ecol[t])];
        // ---- Abar grows: the old columns' new rows, the new columns, ebar's new rows
        // (in half: all of Abar and ebar anew)
        const int ld = lmax;
        const int c0 = q0;                // first column factored in this pass
        const int r0 = HALF ? 0 : nI;     // first row of ebar set in this pass
        const int e0 = Lg;                // first entry scattered in this pass
        for (int t = lane; t < c0 * nnew; t += 32) Ab[(t / nnew) * ld + nI + t % nnew] = 0.0f;
        for (int t = lane; t < (nJ - c0) * nIn; t += 32) Ab[(c0 + t / nIn) * ld + t % nIn] = 0.0f;
        for (int t = r0 + lane; t < nIn; t += 32) cv[t] = 0.0f;
        __syncwarp();
        const int uk = lb_i32(Is, nIn, (int)k);
        const bool k_in = uk < nIn && Is[uk] == (int)k;
        const int pk = k_in ? Ip[uk] : nIn;
        if (lane == 0 && k_in && pk >= r0) cv[pk] = 1.0f;  // ebar's new rows: zero but for k
        float f2 = 0.0f;
        for (int t = e0 + lane; t < Ln; t += 32) {
            Ab[eq[t] * ld + ecol[t]] = eval[t];
            if (!HALF) f2 = F::add(f2, F::mul(eval[t], eval[t]));
        }
        __syncwarp();
        if (HALF) {  // ||Abar||_F column by column, as a fresh factorisation forms it
            for (int t = lane; t < nJ * nIn; t += 32) {
                const float a = Ab[(t / nIn) * ld + t % nIn];
                f2 = F::add(f2, F::mul(a, a));
            }
            fro2 = F::wsum(f2);
        } else {
            fro2 = F::add(fro2, F::wsum(f2));
        }
        nI = nIn;
        L = Ln;
        max_rows = max(max_rows, nI);
        rankdef = nI < nJ;
        const float fro = F::sqrt(fro2);
        // the old reflectors (zero on the new rows) on the new columns
        for (int c = 0; c < c0 && !rankdef; ++c) {
            const float* col_c = Ab + c * ld;
            const float twoinv = tw[c];
            for (int cc = c0; cc < nJ; ++cc) {
                float* tgt = Ab + cc * ld;
                float dot = 0.0f;
                for (int p = c + lane; p < nI; p += 32) dot = F::add(dot, F::mul(col_c[p], tgt[p]));
                dot = F::wsum(dot);
                const float tau = F::mul(dot, twoinv);
                for (int p = c + lane; p < nI; p += 32) tgt[p] = F::sub(tgt[p], F::mul(tau, col_c[p]));
                __syncwarp();
            }
        }
        // Householder QR of the new columns below the old ones, with the sign choice
        // v_1 = x_1 + sign(x_1) ||x||, applied to ebar as well; warp-shuffle reductions
        for (int c = c0; c < nJ && !rankdef; ++c) {
            float* col_c = Ab + c * ld;
            float s2 = 0.0f;
            for (int p = c + lane; p < nI; p += 32) s2 = F::add(s2, F::mul(col_c[p], col_c[p]));
            s2 = F::wsum(s2);
            const float sig = F::sqrt(s2);
            const float x0 = col_c[c];
            if (!(sig > 0.0f)) {
                rankdef = true;
                break;
            }
            const float sgn = x0 >= 0.0f ? 1.0f : -1.0f;
            const float v0 = F::add(x0, sgn * sig);
            const float vtv = F::mul(F::mul(2.0f, sig), F::add(sig, fabsf(x0)));
            const float twoinv = F::div(2.0f, vtv);
            __syncwarp();
            if (lane == 0) {
                col_c[c] = v0;
                tw[c] = twoinv;
            }
            __syncwarp();
            for (int cc = c + 1; cc <= nJ; ++cc) {
                float* tgt = cc < nJ ? Ab + cc * ld : cv;
                float dot = 0.0f;
                for (int p = c + lane; p < nI; p += 32) dot = F::add(dot, F::mul(col_c[p], tgt[p]));
                dot = F::wsum(dot);
                const float tau = F::mul(dot, twoinv);
                for (int p = c + lane; p < nI; p += 32) tgt[p] = F::sub(tgt[p], F::mul(tau, col_c[p]));
                __syncwarp();
            }
            const float rcc = -sgn * sig;
            if (lane == 0) rdiag[c] = rcc;
            if (!(fabsf(rcc) > (float)nI * u_f * fro)) rankdef = true;
        }
        __syncwarp();
        nJ_old = nJ;
        ++solves;
        if (rankdef) break;
        if (lane == 0) {
            for (int c = nJ - 1; c >= 0; --c) {
                float s = cv[c];
                for (int cc = c + 1; cc < nJ; ++cc) s = F::sub(s, F::mul(Ab[cc * ld + c], mv[cc]));
                mv[c] = F::div(s, rdiag[c]);
            }
        }
        __syncwarp();
        // sbar = Abar mbar - ebar from the gathered entries (distinct rows within one q)
        for (int t = lane; t < nI; t += 32) sv[t] = 0.0f;
        __syncwarp();
        if (lane == 0 && k_in) sv[pk] = -1.0f;
        __syncwarp();
        for (int q = 0; q < nJ; ++q) {
            const float mq = mv[q];
            for (int t = eoff[q] + lane; t < eoff[q + 1]; t += 32) {
                const int p = ecol[t];
                sv[p] = F::add(sv[p], F::mul(eval[t], mq));
            }
            __syncwarp();
        }
        float r2 = 0.0f;
        for (int t = lane; t < nI; t += 32) r2 = F::add(r2, F::mul(sv[t], sv[t]));
        r2sum = F::wsum(r2);
        res_norm = F::sqrt(r2sum);
        if (res_norm <= spai_eps) {
            conv = true;
            break;
        }
        if (step == alpha) break;

        // ---- candidates: (union over l in I u {k} of N_l) \ J, each once.  Row l
        // of B lists the j with b_lj != 0 (tcol) and the values (tval), so one
        // sweep over the rows l in I inserts every candidate j into an
        // open-addressing hash table and accumulates sbar^T B(I, j) = sum over l
        // in I of sbar_l b_lj in fixed point (2^-40 units, exact integer sums,
        // independent of the order).  ||B e_j||^2 is precomputed per column.
        // A full table (only possible in the first tier, whose table may have
        // fewer slots than the candidate bound) sends the column to the second.
        const int nL = nI + (k_in ? 0 : 1);
        const int hshift = 32 - (31 - __clz(H));
        bool full = false;
        for (int t = lane; t < nL; t += 32) {
            const int l = t < nI ? I[t] : (int)k;
            const float sl = t < nI ? sv[t] : 0.0f;
            const int e = trp[l + 1];
            for (int p = trp[l]; p < e; ++p) {
                const int j = tcol[p];  // members of J are inserted too and skipped by the scan
                const long long term = fix40(F::mul(sl, tval[p]));
                unsigned h = ((unsigned)j * 0x9E3779B1u) >> hshift;
                int probe = 0;
                for (; probe < H; ++probe) {
                    const int prev = atomicCAS(tab + h, -1, j);
                    if (prev == -1 || prev == j) {
                        atomicAdd(reinterpret_cast<unsigned long long*>(acc + h), (unsigned long long)term);
                        break;
                    }
                    h = (h + 1) & (unsigned)(H - 1);
                }
                if (probe == H) full = true;
            }
        }
        __syncwarp();
        if (__any_sync(0xffffffffu, full)) {  // first tier only: the second's H exceeds every candidate count
            if (redo_list) redo = true;
            else capped = true;
            break;
        }
        // ---- rho per candidate while the table is emptied into keys/rho (in place: a
        // candidate moves to a slot at or below its own, read before any write), and
        // the mean of rho (<= ||sbar|| <= 1) as a fixed-point sum
        int nc = 0;
        long long rsum = 0;
        for (int b0 = 0; b0 < H; b0 += 32) {
            const int v = tab[b0 + lane];
            const bool flag = v >= 0 && !contains(Js, nJ, v);
            float rj = 0.0f;
            long long av = 0;
            if (v >= 0) {
                av = acc[b0 + lane];
                tab[b0 + lane] = -1;
                acc[b0 + lane] = 0;
            }
            if (flag) {
                const float num = F::r(unfix40(av));
                const float den = bnorm2[v];
                float rr = r2sum;
                if (den > 0.0f) rr = F::sub(r2sum, F::div(F::mul(num, num), den));
                rj = F::sqrt(rr > 0.0f ? rr : 0.0f);
                rsum += fix40(rj);
            }
            const unsigned m = __ballot_sync(0xffffffffu, flag);
            if (flag) {
                const int o = nc + __popc(m & ((1u << lane) - 1u));
                keys[o] = v;
                rho[o] = rj;
            }
            nc += __popc(m);
            __syncwarp();
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
        __syncwarp();
        if (nc == 0) break;
        const float mean = F::div(F::r(unfix40(rsum)), (float)nc);
        // ---- up to beta picks: smallest rho (then smaller j) among rho <= mean
        int npick = 0;
        for (int r = 0; r < beta; ++r) {
            float best = INFINITY;
            int bj = INT_MAX, bt = -1;
            for (int t = lane; t < nc; t += 32) {
                const float rv = rho[t];
                const int jv = keys[t];
                if (rv <= mean && (rv < best || (rv == best && jv < bj))) {
                    best = rv;
                    bj = jv;
                    bt = t;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
                const int ot = __shfl_xor_sync(0xffffffffu, bt, o);
                if (ob < best || (ob == best && oj < bj)) {
                    best = ob;
                    bj = oj;
                    bt = ot;
                }
            }
            if (bt < 0) break;
            if (lane == 0) {
                rho[bt] = INFINITY;
                picks[npick] = bj;
            }
            ++npick;
            __syncwarp();
        }
        // the table's storage back to empty for the next pass
        for (int t = lane; t < nc; t += 32) {
            keys[t] = -1;
            acc[t] = 0;
        }
        __syncwarp();
        if (npick == 0) break;
        if (nJ + npick > jmax) {  // only the first tier's jmax is below 1 + alpha beta
            if (redo_list) redo = true;
            else capped = true;
            break;
        }
        // ---- the picks join J (ascending among themselves) and Js
        if (lane == 0) {
            for (int a = 1; a < npick; ++a) {  // insertion sort of the picks
                const int v = picks[a];
                int b = a - 1;
                while (b >= 0 && picks[b] > v) {
                    picks[b + 1] = picks[b];
                    --b;
                }
                picks[b + 1] = v;
            }
            for (int a = 0; a < npick; ++a) {
                if (HALF) {  // J ascending (every pass factors afresh, columns in this order)
                    int b = nJ + a - 1;
                    while (b >= 0 && J[b] > picks[a]) {
                        J[b + 1] = J[b];
                        stp[b + 1] = stp[b];
                        --b;
                    }
                    J[b + 1] = picks[a];
                    stp[b + 1] = step + 1;
                } else {
                    J[nJ + a] = picks[a];
                    stp[nJ + a] = step + 1;
                }
                int b = nJ + a - 1;  // insertion into the sorted copy
                while (b >= 0 && Js[b] > picks[a]) {
                    Js[b + 1] = Js[b];
                    --b;
                }
                Js[b + 1] = picks[a];
            }
        }
        __syncwarp();
        nJ += npick;
    }
    if (redo) {
        if (lane == 0) redo_list[atomicAdd(redo_count, 1)] = (int32_t)k;
        return;
    }
    if (rankdef) res_norm = 1.0f;
    // M[k, J[q]] = mbar_q d_J[q]  (M = M'^T D), the columns in ascending order
    if (lane == 0) {
        for (int a = 1; a < nJ; ++a) {
            const int v = J[a], sa = stp[a];
            const float ma = mv[a];
            int b = a - 1;
            while (b >= 0 && J[b] > v) {
                J[b + 1] = J[b];
                stp[b + 1] = stp[b];
                mv[b + 1] = mv[b];
                --b;
            }
            J[b + 1] = v;
            stp[b + 1] = sa;
            mv[b + 1] = ma;
        }
    }
    __syncwarp();
    for (int q = lane; q < nJ; q += 32) {
        const int j = J[q];
        const int64_t o = (int64_t)q * n + k;
        Jo[o] = j;
        const float m = rankdef ? 0.0f : F::from64(__dmul_rn((double)mv[q], d[j]));
        if (!isfinite(m)) atomicAdd(&cnt->n_nonfinite, 1);
        Mo[o] = m;
        So[o] = (int8_t)stp[q];
    }
    if (lane == 0) {
        nJo[k] = nJ;
        resid[k] = res_norm;
        cinfo[k] = solves | (conv ? 1 << 8 : 0) | (rankdef ? 1 << 9 : 0) | (capped ? 1 << 10 : 0);
        if (conv) atomicAdd(&cnt->n_conv, 1);
        if (rankdef) atomicAdd(&cnt->n_rankdef, 1);
        if (capped) atomicAdd(&cnt->n_capped, 1);
        atomicMax(&cnt->max_cols, nJ);
        atomicMax(&cnt->max_rows, max_rows);
        atomic_max_nonneg(&cnt->max_resid, res_norm);
        atomicAdd(&cnt->solves, (unsigned long long)solves);
    }
}

// per column of A: its entry count (int64, for the scan), and the largest row
__global__ void k_col_counts(int n, const int32_t* __restrict__ arp, const int32_t* __restrict__ acol,
                             unsigned long long* __restrict__ cnt, int* __restrict__ rowmax) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = arp[i], e = arp[i + 1];
    atomicMax(rowmax, e - b);
    for (int p = b; p < e; ++p) atomicAdd(cnt + acol[p], 1ull);
}

__global__ void k_i64_to_i32_rp(int64_t count, const int64_t* __restrict__ in, int32_t* __restrict__ out,
                                int* __restrict__ mx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > count) return;
    out[i] = (int32_t)in[i];
    if (i < count) atomicMax(mx, (int)(in[i + 1] - in[i]));
}

// B = A^T D in u_f: bval[p] = fl_uf(a_p d_i) for the entries p of row i of A
// (column i of B), and bnorm2[i] = ||B e_i||^2 summed in u_f in row order
template <bool HALF>
__global__ void k_bvals(int n, const int32_t* __restrict__ arp, const double* __restrict__ aval,
                        const double* __restrict__ d, float* __restrict__ bval, float* __restrict__ bnorm2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double di = d[i];
    float s2 = 0.0f;
    for (int p = arp[i]; p < arp[i + 1]; ++p) {
        const float b = UfOps<HALF>::from64(__dmul_rn(aval[p], di));
        bval[p] = b;
        s2 = UfOps<HALF>::add(s2, UfOps<HALF>::mul(b, b));
    }
    bnorm2[i] = s2;
}

// the rows of B: row l lists the j with b_lj = a_jl d_j != 0 (the rows of A
// with an entry in column l) and those values; the order within a row is
// irrelevant, every use of a row is order-independent
__global__ void k_tfill(int n, const int32_t* __restrict__ arp, const int32_t* __restrict__ acol,
                        const float* __restrict__ bval, const int32_t* __restrict__ trp, int32_t* __restrict__ cursor,
                        int32_t* __restrict__ tcol, float* __restrict__ tval) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int p = arp[i]; p < arp[i + 1]; ++p) {
        const int c = acol[p];
        const int o = trp[c] + atomicAdd(cursor + c, 1);
        tcol[o] = (int32_t)i;
        tval[o] = bval[p];
    }
}

__global__ void k_counts_i64(int n, const int32_t* __restrict__ nJ, int64_t* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = nJ[i];
}

// the per-column slots (column-major, n per slot) to CSR rows of M
__global__ void k_adaptive_to_csr(int n, const int32_t* __restrict__ Jo, const float* __restrict__ Mo,
                                  const int8_t* __restrict__ So, const int32_t* __restrict__ nJ,
                                  const int32_t* __restrict__ rp, int32_t* __restrict__ col, double* __restrict__ val,
                                  int8_t* __restrict__ st) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int b = rp[k];
    for (int q = 0; q < nJ[k]; ++q) {
        const int64_t o = (int64_t)q * n + k;
        col[b + q] = Jo[o];
        val[b + q] = (double)Mo[o];
        st[b + q] = So[o];
    }
}

}  // namespace bspai

using namespace bspai;

// a CUDA runtime error inside bspai_build_adaptive: release everything, report it
#define ATRY(expr)                                                                   \
    do {                                                                             \
        cudaError_t e_ = (expr);                                                     \
        if (e_ != cudaSuccess) return fail(cuda_error(e_, #expr, __FILE__, __LINE__)); \
    } while (0)

extern "C" {

int bspai_build_adaptive(const bspai_csr_t* A, double spai_eps, int32_t alpha, int32_t beta, int32_t imax_rows,
                         bspai_prec_t u_f, bspai_stream_t st, bspai_M_h* M_out, bspai_build_info_t* info) {
    cudaStream_t s = (cudaStream_t)st;
    if (!M_out) return set_error(BSPAI_ERR_INVALID, "bspai_build_adaptive: null M_out");
    *M_out = nullptr;
    if (!A) return set_error(BSPAI_ERR_INVALID, "bspai_build_adaptive: null matrix");
    if (A->n < 0) return set_error(BSPAI_ERR_INVALID, "bspai_build_adaptive: negative size");
    if (A->n > 0 && (!A->row_ptr || !A->col || !A->val))
        return set_error(BSPAI_ERR_INVALID, "bspai_build_adaptive: missing CSR arrays");
    if (u_f != BSPAI_FP32 && u_f != BSPAI_FP16)
        return set_error(BSPAI_ERR_UNSUPPORTED, "bspai_build_adaptive: u_f must be FP32 or FP16");
    const bool half = u_f == BSPAI_FP16;
    if (!(spai_eps > 0.0)) return set_error(BSPAI_ERR_INVALID, "bspai_build_adaptive: spai_eps must be > 0");
    if (alpha < 0 || alpha > 16 || beta < 0 || beta > 32)
        return set_error(BSPAI_ERR_INVALID, "bspai_build_adaptive: need 0 <= alpha <= 16 and 0 <= beta <= 32");
    if (imax_rows < 1) return set_error(BSPAI_ERR_INVALID, "bspai_build_adaptive: imax_rows must be >= 1");
    BSPAI_TRY(validate_csr(A, true, "bspai_build_adaptive (A)", s));
    const int n = A->n;
    const int jmax = 1 + alpha * beta;
    int second_tier = 0;
    auto* M = new bspai_spai();
    M->magic = kMagicM;
    M->stream = s;
    M->n = n;
    M->uf = u_f;
    double* d = nullptr;
    unsigned long long* ccount = nullptr;
    int64_t* i64 = nullptr;
    int32_t *trp = nullptr, *tcol = nullptr, *cursor = nullptr, *Jo = nullptr, *nJo = nullptr, *cinfo = nullptr;
    int32_t* mcol = nullptr;
    double* mval = nullptr;
    float *bval = nullptr, *bnorm2 = nullptr, *tval = nullptr;
    float* Mo = nullptr;
    int8_t* So = nullptr;
    int* maxes = nullptr;
    AdaptiveCounters* cnt = nullptr;
    auto cleanup = [&]() {
        dfree(d, s);
        dfree(ccount, s);
        dfree(i64, s);
        dfree(trp, s);
        dfree(tcol, s);
        dfree(cursor, s);
        dfree(Jo, s);
        dfree(nJo, s);
        dfree(mcol, s);
        dfree(mval, s);
        dfree(bval, s);
        dfree(bnorm2, s);
        dfree(tval, s);
        dfree(Mo, s);
        dfree(So, s);
        dfree(maxes, s);
        dfree(cnt, s);
    };
    auto fail = [&](int code) {
        cleanup();
        dfree(cinfo, s);
        bspai_free(M);
        return code;
    };
    int rc = BSPAI_OK;
    const size_t n1 = (size_t)n + 1;
    if ((rc = dalloc_t(&maxes, 2, s))) return fail(rc);
    if ((rc = dalloc_t(&cnt, 1, s))) return fail(rc);
    if ((rc = dalloc_t(&M->resid, (size_t)(n > 0 ? n : 1), s))) return fail(rc);
    if ((rc = dalloc_t(&cinfo, (size_t)(n > 0 ? n : 1), s))) return fail(rc);
    ATRY(cudaMemsetAsync(maxes, 0, 2 * sizeof(int), s));
    ATRY(cudaMemsetAsync(cnt, 0, sizeof(AdaptiveCounters), s));
    int hmax[2] = {0, 0};  // largest row of A, largest column of A
    int64_t nnzA = 0;
    if (n > 0) {
        ProfScope ps(BSPAI_K_OTHER, s);
        if ((rc = dalloc_t(&d, (size_t)n, s))) return fail(rc);
        if ((rc = dalloc_t(&ccount, (size_t)n, s))) return fail(rc);
        if ((rc = dalloc_t(&i64, n1, s))) return fail(rc);
        if ((rc = dalloc_t(&trp, n1, s))) return fail(rc);
        if ((rc = dalloc_t(&cursor, (size_t)n, s))) return fail(rc);
        ATRY(cudaMemsetAsync(ccount, 0, sizeof(unsigned long long) * (size_t)n, s));
        ATRY(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)n, s));
        if ((rc = launch_row_absmax_inv(n, A->row_ptr, A->val, d, s))) return fail(rc);
        const unsigned g = (unsigned)ceil_div(n, 256);
        k_col_counts<<<g, 256, 0, s>>>(n, A->row_ptr, A->col, ccount, maxes);
        note_launch();
        if ((rc = scan_exclusive_i64(reinterpret_cast<const int64_t*>(ccount), i64, n, s))) return fail(rc);
        k_i64_to_i32_rp<<<(unsigned)ceil_div((int64_t)n + 1, 256), 256, 0, s>>>(n, i64, trp, maxes + 1);
        note_launch();
        ATRY(cudaMemcpyAsync(&nnzA, i64 + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        ATRY(cudaMemcpyAsync(hmax, maxes, sizeof hmax, cudaMemcpyDeviceToHost, s));
        ATRY(cudaStreamSynchronize(s));
        if ((rc = dalloc_t(&tcol, (size_t)(nnzA > 0 ? nnzA : 1), s))) return fail(rc);
        if ((rc = dalloc_t(&tval, (size_t)(nnzA > 0 ? nnzA : 1), s))) return fail(rc);
        if ((rc = dalloc_t(&bval, (size_t)(nnzA > 0 ? nnzA : 1), s))) return fail(rc);
        if ((rc = dalloc_t(&bnorm2, (size_t)n, s))) return fail(rc);
        (half ? k_bvals<true> : k_bvals<false>)<<<g, 256, 0, s>>>(n, A->row_ptr, A->val, d, bval, bnorm2);
        note_launch();
        k_tfill<<<g, 256, 0, s>>>(n, A->row_ptr, A->col, bval, trp, cursor, tcol, tval);
        note_launch();
        ATRY(cudaGetLastError());
    }
    const int rowmax = hmax[0] > 0 ? hmax[0] : 1;
    const int colmax = hmax[1] > 0 ? hmax[1] : 1;
    if (imax_rows < rowmax)
        return fail(set_error(BSPAI_ERR_INVALID, "bspai_build_adaptive: imax_rows = %d is below the longest row of A (%d)",
                              imax_rows, rowmax));
    // the shadow of jmax rows has at most jmax * rowmax entries
    const int64_t gmax64 = (int64_t)jmax * rowmax;
    const int lmax = (int)(gmax64 < imax_rows ? gmax64 : imax_rows);
    auto pow2_len = [](int64_t need, bool strictly_above) {
        int64_t p = 32;
        while ((strictly_above ? p <= need : p < need) && p < ((int64_t)1 << 26)) p <<= 1;
        return (int)p;
    };
    // the sizes of one tier: |J| <= jm, |I| <= lm; candidates come from the rows
    // of A^T over I u {k} (at most (lm + 1) colmax of them, and at most n)
    struct Tier {
        int jmax, lmax, gmax, lp2, cmax, H, warps;
        size_t per_warp;
    };
    const size_t smem_cap = 200 * 1024;
    auto tier = [&](int jm, int lm, int hcap) {
        Tier t{};
        t.jmax = jm;
        t.lmax = lm;
        t.gmax = jm * rowmax;
        t.lp2 = pow2_len(t.gmax, false);
        const int64_t c = (int64_t)(lm + 1) * colmax;
        t.cmax = (int)(c < n ? c : n);
        t.H = pow2_len(t.cmax, true);  // more slots than candidates: no insertion can fail
        if (hcap > 0 && t.H > hcap) t.H = hcap;  // first tier: a full table reruns the column
        // the table's storage is also the shadow sort's and the row merge's scratch
        if (t.H < t.lp2) t.H = t.lp2;
        if (t.H < lm) t.H = pow2_len(lm, false);
        t.per_warp = adaptive_layout(t.jmax, t.lmax, t.gmax, t.lp2, t.H).total;
        t.warps = 8;
        while (t.warps > 1 && t.per_warp * t.warps > smem_cap) t.warps >>= 1;
        return t;
    };
    const Tier full = tier(jmax, lmax, 0);
    if (full.per_warp * full.warps > smem_cap)
        return fail(set_error(BSPAI_ERR_UNSUPPORTED,
                              "bspai_build_adaptive: one column needs %zu bytes of shared memory (|J| <= %d, |I| <= %d, "
                              "%d candidates); lower alpha, beta or imax_rows",
                              full.per_warp, jmax, lmax, full.cmax));
    // first tier: |J| <= 12, |I| <= 64, 256 candidate slots (when that is smaller
    // and the longest row fits): about 9 KB per column, three blocks of 8 warps per SM
    const Tier small = tier(jmax < 12 ? jmax : 12, lmax < 64 ? lmax : 64, 256);
    const bool two_tier = (small.jmax < jmax || small.lmax < lmax) && rowmax <= small.lmax &&
                          small.per_warp < full.per_warp && small.per_warp * small.warps <= smem_cap;
    const size_t slots = (size_t)jmax * (size_t)(n > 0 ? n : 1);
    if ((rc = dalloc_t(&Jo, slots, s))) return fail(rc);
    if ((rc = dalloc_t(&Mo, slots, s))) return fail(rc);
    if ((rc = dalloc_t(&So, slots, s))) return fail(rc);
    if ((rc = dalloc_t(&nJo, (size_t)(n > 0 ? n : 1), s))) return fail(rc);
    if (n > 0) {
        ProfScope ps(BSPAI_K_SPAI, s);
        const size_t smem_full = full.per_warp * full.warps, smem_s = small.per_warp * small.warps;
        const size_t smem_max = two_tier && smem_s > smem_full ? smem_s : smem_full;
        auto kern = half ? k_spai_adaptive<true> : k_spai_adaptive<false>;
        ATRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
        const float uf = half ? 4.8828125e-04f : 5.9604644775390625e-08f;  // the rank test's unit roundoff
        int nredo = n;
        int32_t* redo = nullptr;  // the columns the second tier runs (all of them without a first tier)
        if (two_tier) {
            // cursor (the redo count) is reused: it was the A^T fill cursor
            if ((rc = dalloc_t(&redo, (size_t)n, s))) return fail(rc);
            ATRY(cudaMemsetAsync(cursor, 0, sizeof(int32_t), s));
            kern<<<(unsigned)ceil_div(n, small.warps), 32 * small.warps, smem_s, s>>>(
                n, n, nullptr, A->row_ptr, A->col, bval, bnorm2, d, trp, tcol, tval, (float)spai_eps, uf, alpha, beta,
                small.jmax,
                small.lmax, small.gmax, small.lp2, small.H, imax_rows, redo, cursor, Jo, Mo, So, nJo,
                M->resid, cinfo, cnt);
            note_launch();
            cudaError_t e = cudaGetLastError();
            if (!e) e = cudaMemcpyAsync(&nredo, cursor, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (!e) e = cudaStreamSynchronize(s);
            if (e) {
                dfree(redo, s);
                return fail(cuda_error(e, "adaptive SPAI first tier", __FILE__, __LINE__));
            }
        }
        if (nredo > 0) {
            kern<<<(unsigned)ceil_div(nredo, full.warps), 32 * full.warps, smem_full, s>>>(
                n, nredo, redo, A->row_ptr, A->col, bval, bnorm2, d, trp, tcol, tval, (float)spai_eps, uf, alpha, beta,
                jmax, lmax,
                full.gmax, full.lp2, full.H, imax_rows, nullptr, nullptr, Jo, Mo, So, nJo, M->resid, cinfo,
                cnt);
            note_launch();
        }
        cudaError_t e = cudaGetLastError();
        dfree(redo, s);
        if (e) return fail(cuda_error(e, "adaptive SPAI", __FILE__, __LINE__));
        second_tier = nredo;
    }
    // CSR of M from the per-column slots, then the SELL form every product uses
    int64_t nnzM = 0;
    if ((rc = dalloc_t(&M->csr_row_ptr, n1, s))) return fail(rc);
    if (n > 0) {
        ProfScope ps(BSPAI_K_OTHER, s);
        const unsigned g = (unsigned)ceil_div(n, 256);
        k_counts_i64<<<g, 256, 0, s>>>(n, nJo, reinterpret_cast<int64_t*>(ccount));
        note_launch();
        if ((rc = scan_exclusive_i64(reinterpret_cast<const int64_t*>(ccount), i64, n, s))) return fail(rc);
        k_i64_to_i32_rp<<<(unsigned)ceil_div((int64_t)n + 1, 256), 256, 0, s>>>(n, i64, M->csr_row_ptr, maxes);
        note_launch();
        ATRY(cudaMemcpyAsync(&nnzM, i64 + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        ATRY(cudaStreamSynchronize(s));
        if ((rc = dalloc_t(&mcol, (size_t)(nnzM > 0 ? nnzM : 1), s))) return fail(rc);
        if ((rc = dalloc_t(&mval, (size_t)(nnzM > 0 ? nnzM : 1), s))) return fail(rc);
        if ((rc = dalloc_t(&M->step_added, (size_t)(nnzM > 0 ? nnzM : 1), s))) return fail(rc);
        k_adaptive_to_csr<<<g, 256, 0, s>>>(n, Jo, Mo, So, nJo, M->csr_row_ptr, mcol, mval, M->step_added);
        note_launch();
        ATRY(cudaGetLastError());
        if ((rc = sell_from_csr(n, M->csr_row_ptr, mcol, mval, &M->sell, nullptr, &M->val, &M->rowlen, s)))
            return fail(rc);
    } else {
        ATRY(cudaMemsetAsync(M->csr_row_ptr, 0, sizeof(int32_t), s));
        if ((rc = sell_from_csr(0, M->csr_row_ptr, nullptr, nullptr, &M->sell, nullptr, &M->val, &M->rowlen, s)))
            return fail(rc);
    }
    M->nnz = nnzM;
    M->col_info = cinfo;
    cinfo = nullptr;
    AdaptiveCounters hc{};
    ATRY(cudaMemcpyAsync(&hc, cnt, sizeof hc, cudaMemcpyDeviceToHost, s));
    ATRY(cudaStreamSynchronize(s));
    cleanup();
    if (info) {
        info->n = n;
        info->max_cols = hc.max_cols;
        info->max_rows = hc.max_rows;
        info->n_converged = hc.n_conv;
        info->n_rank_deficient = hc.n_rankdef;
        info->nnz = nnzM;
        info->max_resid = hc.max_resid;
        info->n_capped = hc.n_capped;
        info->n_second_tier = second_tier;
        info->total_solves = (int64_t)hc.solves;
    }
    *M_out = M;
    if (hc.n_nonfinite > 0) {
        set_error(BSPAI_NONFINITE, "bspai_build_adaptive: %d entries of M overflowed the range of u_f", hc.n_nonfinite);
        return BSPAI_NONFINITE;
    }
    if (hc.n_rankdef > 0) {
        set_error(BSPAI_RANK_DEFICIENT, "bspai_build_adaptive: %d least-squares blocks were rank deficient",
                  hc.n_rankdef);
        return BSPAI_RANK_DEFICIENT;
    }
    return BSPAI_OK;
}

int bspai_M_adaptive_export(bspai_M_h M, int8_t* step_added, int32_t* col_info, bspai_stream_t st) {
    cudaStream_t s = (cudaStream_t)st;
    if (!M || M->magic != kMagicM) return set_error(BSPAI_ERR_INVALID, "bspai_M_adaptive_export: bad handle");
    if (!M->col_info)
        return set_error(BSPAI_ERR_UNSUPPORTED, "bspai_M_adaptive_export: M was not built by bspai_build_adaptive");
    if (step_added && M->nnz > 0)
        CUDA_TRY(cudaMemcpyAsync(step_added, M->step_added, (size_t)M->nnz, cudaMemcpyDeviceToDevice, s));
    if (col_info && M->n > 0)
        CUDA_TRY(cudaMemcpyAsync(col_info, M->col_info, sizeof(int32_t) * (size_t)M->n, cudaMemcpyDeviceToDevice, s));
    return BSPAI_OK;
}

}  // extern "C"
