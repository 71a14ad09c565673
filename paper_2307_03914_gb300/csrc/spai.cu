// spai.cu -- fixed-pattern sparse approximate inverse on the GPU.
//
// Section 2.2 (eq. fronormmin) decouples min ||I - B M'||_F into one small
// least-squares problem per column (eq. redprob); Alg 2.1 with alpha = 0 solves
// each by Householder QR.  Per Section 4 and Alg 3.1, SPAI runs on B = A^T D
// with D = diag(1 / max_i |a_ji|), and the left preconditioner is M = M'^T D,
// so column k of M' is row k of M and column j of B is row j of A times d_j.
//
// One warp per column k, in u_f = fp32:
//   J_k   = pattern of row k of M (ascending)
//   I_k   = shadow: the union of the columns of rows J_k of A, sorted (bitonic
//           sort of the gathered candidates in shared memory, then a
//           ballot/popc compaction of the distinct values)
//   Abar  = B(I_k, J_k) in fp32 (fp64 product a * d_j, rounded once), ebar = e_k(I_k)
//   Householder QR with the sign choice v_1 = x_1 + sign(x_1) ||x||, applied to
//   Abar and ebar; warp-shuffle reductions for every column norm and dot
//   mbar  = R^-1 (Q^T ebar)(1:|J|), by back substitution
//   sbar  = Abar mbar - ebar recomputed from the gathered rows; ||sbar||_2
// and M[k, J_k[q]] = mbar_q d_{J_k[q]} is written into the SELL slots of row k.
#include <climits>

#include "common.cuh"

namespace bspai {

__global__ void k_row_absmax_inv(int n, const int32_t* __restrict__ row_ptr, const double* __restrict__ val,
                                 double* __restrict__ d) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double mx = 0.0;
    for (int p = row_ptr[j]; p < row_ptr[j + 1]; ++p) mx = fmax(mx, fabs(val[p]));
    d[j] = mx > 0.0 ? 1.0 / mx : 1.0;
}

int launch_row_absmax_inv(int n, const int32_t* row_ptr, const double* val, double* d, cudaStream_t s) {
    if (n <= 0) return BSPAI_OK;
    k_row_absmax_inv<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, row_ptr, val, d);
    note_launch();
    CUDA_LAUNCH_CHECK();
    return BSPAI_OK;
}

// per column: |J_k| and the candidate count sum_{j in J_k} |row j of A|
__global__ void __launch_bounds__(256) k_spai_sizes(int n, const int64_t* __restrict__ msptr, const int32_t* __restrict__ mcol,
                             const int32_t* __restrict__ mrowlen, const int32_t* __restrict__ arp,
                             int* __restrict__ out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int nJ = 0, L = 0;
    if (k < n) {
        nJ = mrowlen[k];
        const int64_t base = msptr[k >> 5] + (k & 31);
        for (int q = 0; q < nJ; ++q) {
            const int j = mcol[base + (int64_t)q * kSlice];
            L += arp[j + 1] - arp[j];
        }
    }
    // the warp's maxima, then the block's, then one atomic each
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nJ = max(nJ, __shfl_xor_sync(0xffffffffu, nJ, o));
        L = max(L, __shfl_xor_sync(0xffffffffu, L, o));
    }
    __shared__ int s_nj[8], s_l[8];
    auto mx = [](int a, int b) { return a > b ? a : b; };
    nJ = block_combine(nJ, 0, s_nj, mx);
    L = block_combine(L, 0, s_l, mx);
    if (threadIdx.x == 0) {
        atomicMax(out, nJ);
        atomicMax(out + 1, L);
    }
}

struct SpaiCounters {
    int n_conv;
    int n_rankdef;
    float max_resid;
    int n_nonfinite;  // entries of M outside the range of u_f (fp16: |m| >= 65520 rounds to Inf)
};

// Shared memory of one warp (bytes): dJ (fp64, |J|), J, mbar, R's diagonal,
// A's row start and the entry offset of every j in J (int32, |J| + 1), the
// sort buffer (lp2), I, Abar (|I| x |J|), ebar / Q^T ebar, sbar, and per
// gathered entry its column (then its position in I), scaled value and q.
__host__ __device__ __forceinline__ size_t spai_warp_bytes(int jmax, int lmax, int lp2) {
    return ((size_t)jmax * 8 + (size_t)jmax * 4 * 4 + (size_t)(jmax + 1) * 4 + (size_t)lp2 * 4 +
            (size_t)lmax * 4 + (size_t)lmax * jmax * 4 + (size_t)lmax * 4 * 2 + (size_t)lmax * 4 * 3 + 15) &
           ~(size_t)15;
}

constexpr int kRegJ = 8;  // |J| up to which the register-resident QR path applies

__device__ __forceinline__ int lower_bound_i32(const int* a, int n, int v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// at most 51 registers (five 256-thread blocks per SM): the half instance would
// otherwise take 60 and fit only four
template <bool H>
__global__ void __launch_bounds__(256, 5) k_spai(int n, const int32_t* __restrict__ arp, const int32_t* __restrict__ acol,
                                               const double* __restrict__ aval, const double* __restrict__ d,
                                               const int64_t* __restrict__ msptr, const int32_t* __restrict__ mcol,
                                               const int32_t* __restrict__ mrowlen, float* __restrict__ mval,
                                               float* __restrict__ resid, float spai_eps, float u_f, int jmax,
                                               int lmax, int lp2, SpaiCounters* __restrict__ cnt) {
    using F = UfOps<H>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (k >= n) return;

    // per-warp shared-memory carve-up
    const size_t per_warp = spai_warp_bytes(jmax, lmax, lp2);
    unsigned char* base = smem + per_warp * wib;
    double* dJ = reinterpret_cast<double*>(base);
    int* J = reinterpret_cast<int*>(dJ + jmax);
    float* mv = reinterpret_cast<float*>(J + jmax);
    float* rdiag = mv + jmax;
    int* rbeg = reinterpret_cast<int*>(rdiag + jmax);
    int* eoff = rbeg + jmax;
    int* cand = eoff + jmax + 1;
    int* I = cand + lp2;
    float* Ab = reinterpret_cast<float*>(I + lmax);
    float* cv = Ab + (size_t)lmax * jmax;
    float* sv = cv + lmax;
    int* ecol = reinterpret_cast<int*>(sv + lmax);
    float* eval = reinterpret_cast<float*>(ecol + lmax);
    int* eq = reinterpret_cast<int*>(eval + lmax);

    // J, d_J and the bounds of rows J of A, all loads in one round
    const int nJ = mrowlen[k];
    const int64_t mbase = msptr[k >> 5] + (k & 31);
    for (int q = lane; q < nJ; q += 32) {
        const int j = mcol[mbase + (int64_t)q * kSlice];
        J[q] = j;
        dJ[q] = d[j];
        const int rb = arp[j];
        rbeg[q] = rb;
        eoff[q] = arp[j + 1] - rb;
    }
    __syncwarp();
    if (lane == 0) {
        int acc = 0;
        for (int q = 0; q < nJ; ++q) {
            const int len = eoff[q];
            eoff[q] = acc;
            acc += len;
        }
        eoff[nJ] = acc;
    }
    __syncwarp();
    const int L = eoff[nJ];
    // every entry of rows J of A, gathered at once: its column, its value
    // scaled by d_j and rounded to u_f (the entries of Abar), and its q
    for (int t = lane; t < L; t += 32) {
        int lo = 0, hi = nJ;  // the q with eoff[q] <= t < eoff[q + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (eoff[mid] <= t) lo = mid;
            else hi = mid;
        }
        const int e = rbeg[lo] + (t - eoff[lo]);
        const int c = acol[e];
        ecol[t] = c;
        cand[t] = c;
        eval[t] = F::from64(__dmul_rn(aval[e], dJ[lo]));
        eq[t] = lo;
    }
    int LP = 2;
    while (LP < L) LP <<= 1;
    for (int t = L + lane; t < LP; t += 32) cand[t] = INT_MAX;
    __syncwarp();
    // bitonic sort of cand[0, LP)
    for (int size = 2; size <= LP; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < (LP >> 1); t += 32) {
                const int i = ((t & ~(stride - 1)) << 1) | (t & (stride - 1));  // stride is a power of two
                const int jj = i + stride;
                const bool asc = (i & size) == 0;
                const int a = cand[i], b = cand[jj];
                if ((a > b) == asc) {
                    cand[i] = b;
                    cand[jj] = a;
                }
            }
            __syncwarp();
        }
    }
    // distinct values -> I (sorted)
    int nI = 0;
    for (int b0 = 0; b0 < L; b0 += 32) {
        const int t = b0 + lane;
        const int v = t < L ? cand[t] : INT_MAX;
        const int prev = (t > 0 && t < L) ? cand[t - 1] : -1;
        const bool flag = t < L && v != prev;
        const unsigned m = __ballot_sync(0xffffffffu, flag);
        if (flag) I[nI + __popc(m & ((1u << lane) - 1u))] = v;
        nI += __popc(m);
    }
    __syncwarp();

    bool rankdef = (nJ > 0 && nI < nJ);
    float res_norm = 1.0f;
    if (nJ > 0 && !rankdef && nI <= 32 && nJ <= kRegJ) {
        // Small block (|I| <= 32, |J| <= 8): lane p holds row p of Abar, of
        // Q^T ebar and of the original Abar in registers, so the Householder
        // steps need no shared-memory traffic: the same algorithm as below.
        for (int t = lane; t < nJ * nI; t += 32) Ab[t] = 0.0f;
        __syncwarp();
        const int pk = lower_bound_i32(I, nI, (int)k);
        const bool k_in = pk < nI && I[pk] == (int)k;
        for (int t = lane; t < L; t += 32) Ab[eq[t] * nI + lower_bound_i32(I, nI, ecol[t])] = eval[t];
        __syncwarp();
        const bool mine = lane < nI;
        float a[kRegJ], a0[kRegJ];
#pragma unroll
        for (int q = 0; q < kRegJ; ++q) {
            a[q] = (mine && q < nJ) ? Ab[q * nI + lane] : 0.0f;
            a0[q] = a[q];
        }
        float cvp = (k_in && lane == pk) ? 1.0f : 0.0f;
        float fro = 0.0f;
#pragma unroll
        for (int q = 0; q < kRegJ; ++q) fro = F::add(fro, F::mul(a[q], a[q]));
        fro = F::sqrt(F::wsum(fro));
        float rd[kRegJ];
#pragma unroll
        for (int c = 0; c < kRegJ; ++c) {
            rd[c] = 1.0f;
            if (c >= nJ || rankdef) continue;
            const bool act = mine && lane >= c;
            const float xc = act ? a[c] : 0.0f;
            const float sig = F::sqrt(F::wsum(F::mul(xc, xc)));
            const float x0 = __shfl_sync(0xffffffffu, a[c], c);
            if (!(sig > 0.0f)) {
                rankdef = true;
                continue;
            }
            const float sgn = x0 >= 0.0f ? 1.0f : -1.0f;
            const float v0 = F::add(x0, sgn * sig);
            const float vtv = F::mul(F::mul(2.0f, sig), F::add(sig, fabsf(x0)));
            const float twoinv = F::div(2.0f, vtv);
            const float vp = act ? (lane == c ? v0 : a[c]) : 0.0f;  // reflector v, entries c..|I|-1
#pragma unroll
            for (int cc = c + 1; cc < kRegJ; ++cc) {
                if (cc >= nJ) break;
                const float tau = F::mul(F::wsum(F::mul(vp, a[cc])), twoinv);
                if (act) a[cc] = F::sub(a[cc], F::mul(tau, vp));
            }
            {
                const float tau = F::mul(F::wsum(F::mul(vp, cvp)), twoinv);
                if (act) cvp = F::sub(cvp, F::mul(tau, vp));
            }
            rd[c] = -sgn * sig;
            if (!(fabsf(rd[c]) > (float)nI * u_f * fro)) rankdef = true;
        }
        if (!rankdef) {
            // back substitution R mbar = (Q^T ebar)(1:|J|): lane c holds row c of R
            float m[kRegJ];
#pragma unroll
            for (int q = 0; q < kRegJ; ++q) m[q] = 0.0f;
#pragma unroll
            for (int c = kRegJ - 1; c >= 0; --c) {
                if (c >= nJ) continue;
                float sum = cvp;
#pragma unroll
                for (int cc = c + 1; cc < kRegJ; ++cc)
                    if (cc < nJ) sum = F::sub(sum, F::mul(a[cc], m[cc]));
                m[c] = __shfl_sync(0xffffffffu, F::div(sum, rd[c]), c);
            }
            // sbar = Abar mbar - ebar from the original rows
            float sp = (k_in && lane == pk) ? -1.0f : 0.0f;
#pragma unroll
            for (int q = 0; q < kRegJ; ++q)
                if (q < nJ) sp = F::add(sp, F::mul(a0[q], m[q]));
            res_norm = F::sqrt(F::wsum(mine ? F::mul(sp, sp) : 0.0f));
            if (lane < nJ) {
                float mq = 0.0f;
#pragma unroll
                for (int q = 0; q < kRegJ; ++q)
                    if (q == lane) mq = m[q];
                mv[lane] = mq;
            }
            __syncwarp();
        }
    } else if (nJ > 0 && !rankdef) {
        // Abar (column-major, leading dimension nI) and ebar
        for (int t = lane; t < nJ * nI; t += 32) Ab[t] = 0.0f;
        for (int t = lane; t < nI; t += 32) cv[t] = 0.0f;
        __syncwarp();
        const int pk = lower_bound_i32(I, nI, (int)k);
        const bool k_in = pk < nI && I[pk] == (int)k;
        if (lane == 0 && k_in) cv[pk] = 1.0f;
        for (int t = lane; t < L; t += 32) {
            const int p = lower_bound_i32(I, nI, ecol[t]);
            ecol[t] = p;  // from here on: the entry's row in Abar
            Ab[eq[t] * nI + p] = eval[t];
        }
        __syncwarp();
        float fro = 0.0f;
        for (int t = lane; t < nJ * nI; t += 32) fro = F::add(fro, F::mul(Ab[t], Ab[t]));
        fro = F::sqrt(F::wsum(fro));

        // Householder QR of Abar, applied to ebar as well
        for (int c = 0; c < nJ && !rankdef; ++c) {
            float* col_c = Ab + c * nI;
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
            __syncwarp();
            if (lane == 0) col_c[c] = v0;
            __syncwarp();
            for (int cc = c + 1; cc <= nJ; ++cc) {
                float* tgt = cc < nJ ? Ab + cc * nI : cv;  // the last pass applies the reflector to ebar
                float dot = 0.0f;
                for (int p = c + lane; p < nI; p += 32) dot = F::add(dot, F::mul(col_c[p], tgt[p]));
                dot = F::wsum(dot);
                const float tau = F::div(F::mul(2.0f, dot), vtv);
                for (int p = c + lane; p < nI; p += 32) tgt[p] = F::sub(tgt[p], F::mul(tau, col_c[p]));
                __syncwarp();
            }
            const float rcc = -sgn * sig;
            if (lane == 0) rdiag[c] = rcc;
            if (!(fabsf(rcc) > (float)nI * u_f * fro)) rankdef = true;
        }
        __syncwarp();
        if (!rankdef) {
            // back substitution R mbar = (Q^T ebar)(1:|J|)
            if (lane == 0) {
                for (int c = nJ - 1; c >= 0; --c) {
                    float s = cv[c];
                    for (int cc = c + 1; cc < nJ; ++cc) s = F::sub(s, F::mul(Ab[cc * nI + c], mv[cc]));
                    mv[c] = F::div(s, rdiag[c]);
                }
            }
            __syncwarp();
            // sbar = Abar mbar - ebar, from the original gathered entries
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
            res_norm = F::sqrt(F::wsum(r2));
        }
    }
    if (rankdef) res_norm = 1.0f;
    // M[k, J[q]] = mbar_q d_J[q]  (M = M'^T D)
    for (int q = lane; q < nJ; q += 32) {
        const float m = rankdef ? 0.0f : F::from64(__dmul_rn((double)mv[q], dJ[q]));
        if (!isfinite(m)) atomicAdd(&cnt->n_nonfinite, 1);
        mval[mbase + (int64_t)q * kSlice] = m;
    }
    if (lane == 0) {
        resid[k] = res_norm;
        if (res_norm <= spai_eps) atomicAdd(&cnt->n_conv, 1);
        if (rankdef) atomicAdd(&cnt->n_rankdef, 1);
        atomic_max_nonneg(&cnt->max_resid, res_norm);
    }
}

// fp64 values rounded once to fp16 (held in fp64), for an M imported in u_f = fp16
__global__ void k_round_f16_of_f64(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (double)__half2float(__double2half(x[i]));
}

__global__ void k_sell_to_csr_f32(int n, const int64_t* __restrict__ sptr, const int32_t* __restrict__ scol,
                                  const float* __restrict__ sval, const int32_t* __restrict__ rowlen,
                                  const int32_t* __restrict__ row_ptr, int32_t* __restrict__ col,
                                  float* __restrict__ val) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t b = sptr[r >> 5] + (r & 31);
    const int len = rowlen[r];
    const int o = row_ptr[r];
    for (int l = 0; l < len; ++l) {
        if (col) col[o + l] = scol[b + (int64_t)l * kSlice];
        if (val) val[o + l] = sval[b + (int64_t)l * kSlice];
    }
}

}  // namespace bspai

using namespace bspai;

extern "C" {

int bspai_build(const bspai_csr_t* A, const bspai_csr_t* P, double spai_eps, bspai_prec_t u_f,
                bspai_stream_t st, bspai_M_h* M_out, bspai_build_info_t* info) {
    cudaStream_t s = (cudaStream_t)st;
    if (!M_out) return set_error(BSPAI_ERR_INVALID, "bspai_build: null M_out");
    *M_out = nullptr;
    if (!A || !P) return set_error(BSPAI_ERR_INVALID, "bspai_build: null matrix");
    if (A->n != P->n || A->n < 0) return set_error(BSPAI_ERR_INVALID, "bspai_build: A and pattern sizes differ");
    if (A->n > 0 && (!A->row_ptr || !A->col || !A->val || !P->row_ptr || !P->col))
        return set_error(BSPAI_ERR_INVALID, "bspai_build: missing CSR arrays");
    if (u_f != BSPAI_FP32 && u_f != BSPAI_FP16)
        return set_error(BSPAI_ERR_UNSUPPORTED, "bspai_build: u_f must be FP32 or FP16");
    if (!(spai_eps > 0.0)) return set_error(BSPAI_ERR_INVALID, "bspai_build: spai_eps must be > 0");
    BSPAI_TRY(validate_csr(A, true, "bspai_build (A)", s));
    BSPAI_TRY(validate_csr(P, false, "bspai_build (pattern)", s));
    const int n = A->n;
    auto* M = new bspai_spai();
    M->magic = kMagicM;
    M->stream = s;
    M->n = n;
    M->nnz = P->nnz;
    M->uf = u_f;
    double* d = nullptr;
    int* sizes = nullptr;
    SpaiCounters* cnt = nullptr;
    int st_ = BSPAI_OK;
    auto fail = [&](int code) {
        dfree(d, s);
        dfree(sizes, s);
        dfree(cnt, s);
        bspai_free(M);
        return code;
    };
    {
        ProfScope ps(BSPAI_K_OTHER, s);
        st_ = sell_from_csr(n, P->row_ptr, P->col, nullptr, &M->sell, nullptr, nullptr, &M->rowlen, s);
        if (st_) return fail(st_);
        if ((st_ = dalloc_t(&M->csr_row_ptr, (size_t)n + 1, s))) return fail(st_);
        if ((st_ = dalloc_t(&M->val, (size_t)M->sell.slots, s))) return fail(st_);
        if ((st_ = dalloc_t(&M->resid, (size_t)n, s))) return fail(st_);
        if ((st_ = dalloc_t(&d, (size_t)n, s))) return fail(st_);
        if ((st_ = dalloc_t(&sizes, 2, s))) return fail(st_);
        if ((st_ = dalloc_t(&cnt, 1, s))) return fail(st_);
        cudaError_t e = cudaMemcpyAsync(M->csr_row_ptr, P->row_ptr, sizeof(int32_t) * ((size_t)n + 1),
                                        cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(M->val, 0, sizeof(float) * (size_t)M->sell.slots, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(sizes, 0, 2 * sizeof(int), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(SpaiCounters), s);
        if (e != cudaSuccess) return fail(cuda_error(e, "bspai_build setup", __FILE__, __LINE__));
        if (n > 0) {
            k_row_absmax_inv<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, A->row_ptr, A->val, d);
            note_launch();
            k_spai_sizes<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, M->sell.sptr, M->sell.col, M->rowlen,
                                                                    A->row_ptr, sizes);
            note_launch();
            e = cudaGetLastError();
            if (e != cudaSuccess) return fail(cuda_error(e, "spai sizes", __FILE__, __LINE__));
        }
    }
    int hs[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(hs, sizes, sizeof hs, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(cuda_error(e, "spai sizes copy", __FILE__, __LINE__));
    const int jmax = hs[0] > 0 ? hs[0] : 1;
    const int lmax = hs[1] > 0 ? hs[1] : 1;
    int lp2 = 32;
    while (lp2 < lmax) lp2 <<= 1;
    const size_t per_warp = spai_warp_bytes(jmax, lmax, lp2);
    const size_t smem_cap = 200 * 1024;
    int warps = 8;
    while (warps > 1 && per_warp * warps > smem_cap) warps >>= 1;
    if (per_warp * warps > smem_cap)
        return fail(set_error(BSPAI_ERR_UNSUPPORTED,
                              "bspai_build: least-squares blocks too large (|J| <= %d, candidates <= %d need %zu bytes)",
                              jmax, lmax, per_warp));
    const size_t smem = per_warp * warps;
    if (n > 0) {
        ProfScope ps(BSPAI_K_SPAI, s);
        const bool h = u_f == BSPAI_FP16;
        e = cudaFuncSetAttribute(h ? k_spai<true> : k_spai<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return fail(cuda_error(e, "spai smem attribute", __FILE__, __LINE__));
        // u_f: 2^-24 (fp32) or 2^-11 (fp16), the rank test's unit roundoff
        (h ? k_spai<true> : k_spai<false>)<<<(unsigned)ceil_div(n, warps), 32 * warps, smem, s>>>(
            n, A->row_ptr, A->col, A->val, d, M->sell.sptr, M->sell.col, M->rowlen, M->val, M->resid,
            (float)spai_eps, h ? 4.8828125e-04f : 5.9604644775390625e-08f, jmax, lmax, lp2, cnt);
        note_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(cuda_error(e, "k_spai", __FILE__, __LINE__));
    }
    SpaiCounters hc{};
    e = cudaMemcpyAsync(&hc, cnt, sizeof hc, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(cuda_error(e, "spai counters", __FILE__, __LINE__));
    dfree(d, s);
    dfree(sizes, s);
    dfree(cnt, s);
    if (info) {
        info->n = n;
        info->max_cols = hs[0];
        info->max_rows = hs[1];
        info->n_converged = hc.n_conv;
        info->n_rank_deficient = hc.n_rankdef;
        info->nnz = P->nnz;
        info->max_resid = hc.max_resid;
        info->n_capped = 0;
        info->n_second_tier = 0;
        info->total_solves = n;
    }
    *M_out = M;
    if (hc.n_nonfinite > 0) {
        set_error(BSPAI_NONFINITE, "bspai_build: %d entries of M overflowed the range of u_f", hc.n_nonfinite);
        return BSPAI_NONFINITE;
    }
    if (hc.n_rankdef > 0) {
        set_error(BSPAI_RANK_DEFICIENT, "bspai_build: %d least-squares blocks were rank deficient", hc.n_rankdef);
        return BSPAI_RANK_DEFICIENT;
    }
    return BSPAI_OK;
}

int bspai_M_create(const bspai_csr_t* Mcsr, bspai_prec_t u_f, bspai_stream_t st, bspai_M_h* M_out) {
    cudaStream_t s = (cudaStream_t)st;
    if (!M_out) return set_error(BSPAI_ERR_INVALID, "bspai_M_create: null M_out");
    *M_out = nullptr;
    if (u_f != BSPAI_FP32 && u_f != BSPAI_FP16)
        return set_error(BSPAI_ERR_UNSUPPORTED, "bspai_M_create: u_f must be FP32 or FP16");
    BSPAI_TRY(validate_csr(Mcsr, true, "bspai_M_create", s));
    const int n = Mcsr->n;
    auto* M = new bspai_spai();
    M->magic = kMagicM;
    M->stream = s;
    M->n = n;
    M->nnz = Mcsr->nnz;
    M->uf = u_f;
    int rc = BSPAI_OK;
    {
        ProfScope ps(BSPAI_K_OTHER, s);
        // fp16: round the fp64 values once to fp16 first; the fp32 copy below is then exact
        double* v16 = nullptr;
        if (u_f == BSPAI_FP16 && Mcsr->nnz > 0) {
            rc = dalloc_t(&v16, (size_t)Mcsr->nnz, s);
            if (!rc) {
                k_round_f16_of_f64<<<(unsigned)ceil_div(Mcsr->nnz, 256), 256, 0, s>>>(Mcsr->nnz, Mcsr->val, v16);
                note_launch();
                cudaError_t e = cudaGetLastError();
                if (e) rc = cuda_error(e, "k_round_f16_of_f64", __FILE__, __LINE__);
            }
        }
        if (!rc)
            rc = sell_from_csr(n, Mcsr->row_ptr, Mcsr->col, v16 ? v16 : Mcsr->val, &M->sell, nullptr, &M->val,
                               &M->rowlen, s);
        dfree(v16, s);
        if (!rc) rc = dalloc_t(&M->csr_row_ptr, (size_t)n + 1, s);
        if (!rc) rc = dalloc_t(&M->resid, (size_t)(n > 0 ? n : 1), s);
        if (!rc) {
            cudaError_t e = cudaMemcpyAsync(M->csr_row_ptr, Mcsr->row_ptr, sizeof(int32_t) * ((size_t)n + 1),
                                            cudaMemcpyDeviceToDevice, s);
            if (!e) e = cudaMemsetAsync(M->resid, 0, sizeof(float) * (size_t)(n > 0 ? n : 1), s);
            if (e) rc = cuda_error(e, "bspai_M_create", __FILE__, __LINE__);
        }
    }
    if (rc) {
        bspai_free(M);
        return rc;
    }
    *M_out = M;
    return BSPAI_OK;
}

int bspai_M_export(bspai_M_h M, int32_t* row_ptr, int32_t* col, float* val, float* resid, bspai_stream_t st) {
    cudaStream_t s = (cudaStream_t)st;
    if (!M || M->magic != kMagicM) return set_error(BSPAI_ERR_INVALID, "bspai_M_export: bad handle");
    if (row_ptr)
        CUDA_TRY(cudaMemcpyAsync(row_ptr, M->csr_row_ptr, sizeof(int32_t) * ((size_t)M->n + 1),
                                 cudaMemcpyDeviceToDevice, s));
    if (resid) CUDA_TRY(cudaMemcpyAsync(resid, M->resid, sizeof(float) * (size_t)M->n, cudaMemcpyDeviceToDevice, s));
    if ((col || val) && M->n > 0) {
        k_sell_to_csr_f32<<<(unsigned)ceil_div(M->n, 256), 256, 0, s>>>(M->n, M->sell.sptr, M->sell.col, M->val,
                                                                        M->rowlen, M->csr_row_ptr, col, val);
        note_launch();
        CUDA_LAUNCH_CHECK();
    }
    return BSPAI_OK;
}

}  // extern "C"
