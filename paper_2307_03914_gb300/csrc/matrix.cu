// matrix.cu -- A on the GPU: CSR -> SELL-32 conversion, ||A||_inf, and the
// residual r = b - A x with u_r ~ u^2 (Dot2; Alg 3.1 residual line).
#include <cstdint>

#include "common.cuh"

namespace bspai {

// width of each 32-row slice (max row length), times 32
__global__ void __launch_bounds__(256) k_slice_width(int n, const int32_t* __restrict__ row_ptr,
                                                     int64_t* __restrict__ w) {
    __shared__ int s_len[8];
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nsl = ceil_div(n, kSlice);
    int len = r < n ? row_ptr[r + 1] - row_ptr[r] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
    if ((r & 31) == 0 && r < nsl * kSlice) w[r >> 5] = (int64_t)len * kSlice;
    // the overall width: the block's maximum, one atomic per block
    len = block_combine(len, 0, s_len, [](int a, int b) { return a > b ? a : b; });
    if (threadIdx.x == 0 && len > 0)
        atomicMax(reinterpret_cast<unsigned long long*>(w + nsl), (unsigned long long)len);
}

// scatter the CSR rows into their slices; padding slots get column -1, value 0
__global__ void k_sell_fill(int n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const double* __restrict__ val, const int64_t* __restrict__ sptr,
                            int32_t* __restrict__ scol, double* __restrict__ v64, float* __restrict__ v32,
                            int32_t* __restrict__ rowlen) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nsl = ceil_div(n, kSlice);
    if (r >= nsl * kSlice) return;
    const int64_t s = r >> 5;
    const int lane = (int)(r & 31);
    const int64_t base = sptr[s];
    const int width = (int)((sptr[s + 1] - base) / kSlice);
    int b = 0, len = 0;
    if (r < n) {
        b = row_ptr[r];
        len = row_ptr[r + 1] - b;
    }
    for (int l = 0; l < width; ++l) {
        const int64_t slot = base + (int64_t)l * kSlice + lane;
        if (l < len) {
            scol[slot] = col[b + l];
            if (val) {
                double a = val[b + l];
                if (v64) v64[slot] = a;
                if (v32) v32[slot] = __double2float_rn(a);
            }
        } else {
            scol[slot] = -1;
            if (v64) v64[slot] = 0.0;
            if (v32) v32[slot] = 0.0f;
        }
    }
    if (rowlen && r < n) rowlen[r] = len;
}

int sell_from_csr(int n, const int32_t* row_ptr, const int32_t* col, const double* val, Sell* out,
                  double** val64, float** val32, int32_t** rowlen, cudaStream_t s) {
    Sell S;
    S.n = n;
    S.nslices = (int32_t)ceil_div(n, kSlice);
    int64_t* w = nullptr;
    BSPAI_TRY(dalloc_t(&w, (size_t)S.nslices + 1, s));
    BSPAI_TRY(dalloc_t(&S.sptr, (size_t)S.nslices + 1, s));
    const int64_t rows = (int64_t)S.nslices * kSlice;
    const unsigned grid = (unsigned)ceil_div(rows, 256);
    CUDA_TRY(cudaMemsetAsync(w + S.nslices, 0, sizeof(int64_t), s));  // widest slice (rows per slot)
    if (n > 0) {
        k_slice_width<<<grid, 256, 0, s>>>(n, row_ptr, w);
        note_launch();
        CUDA_LAUNCH_CHECK();
    }
    BSPAI_TRY(scan_exclusive_i64(w, S.sptr, S.nslices, s));
    int64_t wmax = 0;
    CUDA_TRY(cudaMemcpyAsync(&S.slots, S.sptr + S.nslices, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(&wmax, w + S.nslices, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    S.maxw = (int32_t)wmax;
    dfree(w, s);
    BSPAI_TRY(dalloc_t(&S.col, (size_t)S.slots, s));
    double* v64 = nullptr;
    float* v32 = nullptr;
    int32_t* rl = nullptr;
    if (val64) BSPAI_TRY(dalloc_t(&v64, (size_t)S.slots, s));
    if (val32) BSPAI_TRY(dalloc_t(&v32, (size_t)S.slots, s));
    if (rowlen) BSPAI_TRY(dalloc_t(&rl, (size_t)n, s));
    if (n > 0) {
        k_sell_fill<<<grid, 256, 0, s>>>(n, row_ptr, col, val, S.sptr, S.col, v64, v32, rl);
        note_launch();
        CUDA_LAUNCH_CHECK();
    }
    *out = S;
    if (val64) *val64 = v64;
    if (val32) *val32 = v32;
    if (rowlen) *rowlen = rl;
    return BSPAI_OK;
}

// ------------------------------------------------ packed copy for A v in u_p
// A's values rounded to fp32 in the packed slot arrangement (groups of four
// slots per row, see Sell), with 16-bit column differences when every
// |c - r| fits: the layout the vector-load SpMV kernel reads.

// slice widths rounded up to four slots (times 32) and max |c - r| over the entries
__global__ void k_packed_widths(int n, int nsl, const int64_t* __restrict__ sptr, const int32_t* __restrict__ col,
                                int64_t* __restrict__ w, unsigned* __restrict__ dmax, int* __restrict__ wmin) {
    __shared__ unsigned s_dm[8];
    __shared__ int s_wm[8];
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = r < (int64_t)nsl * kSlice;  // whole warps
    const int64_t s = r >> 5;
    const int width = live ? (int)((sptr[s + 1] - sptr[s]) >> 5) : 0;
    unsigned dm = 0;
    if (r < n)
        for (int l = 0; l < width; ++l) {
            const int c = col[sptr[s] + ((int64_t)l << 5) + (r & 31)];
            if (c < 0) continue;
            const int64_t d = (int64_t)c - r;
            const unsigned ad = (unsigned)(d < 0 ? -d : d);
            dm = ad > dm ? ad : dm;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned t = __shfl_xor_sync(0xffffffffu, dm, o);
        dm = t > dm ? t : dm;
    }
    const int pw = (width + 3) & ~3;
    if ((r & 31) == 0 && live) w[s] = (int64_t)pw * kSlice;
    // the block's maximum distance and minimum width, one atomic each per block
    dm = block_combine(dm, 0u, s_dm, [](unsigned a, unsigned b) { return a > b ? a : b; });
    const int wm = block_combine(live ? pw : 0x7fffffff, 0x7fffffff, s_wm, [](int a, int b) { return a < b ? a : b; });
    if (threadIdx.x == 0) {
        if (dm) atomicMax(dmax, dm);
        atomicMin(wmin, wm);
    }
}

__global__ void k_packed_fill(int n, int nsl, const int64_t* __restrict__ sptr, const int32_t* __restrict__ col,
                              const float* __restrict__ val, const int64_t* __restrict__ psptr,
                              int32_t* __restrict__ pcol, int16_t* __restrict__ pcol16, float* __restrict__ pval) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (int64_t)nsl * kSlice) return;
    const int64_t s = r >> 5;
    const int lane = (int)(r & 31);
    const int width = (int)((sptr[s + 1] - sptr[s]) >> 5);
    const int pwidth = (int)((psptr[s + 1] - psptr[s]) >> 5);
    for (int l = 0; l < pwidth; ++l) {
        int c = -1;
        float v = 0.0f;
        if (r < n && l < width) {
            const int64_t sp = sptr[s] + ((int64_t)l << 5) + lane;
            c = col[sp];
            if (c >= 0) v = val[sp];
        }
        const int64_t dp = sell_slot(psptr[s], lane, l, 1);
        if (pcol16) pcol16[dp] = c < 0 ? kCol16Pad : (int16_t)(c - r);
        else pcol[dp] = c;
        pval[dp] = c < 0 ? 0.0f : v;
    }
}

int sell_packed_copy(const Sell& S, const float* val, Sell* out, float** pval, cudaStream_t s) {
    Sell P;
    P.n = S.n;
    P.nslices = S.nslices;
    P.packed = 1;
    int64_t* w = nullptr;
    unsigned* dmax = nullptr;  // dmax[0]: max |c - r|; dmax[1]: narrowest packed width
    auto done = [&](int code) {
        dfree(w, s);
        dfree(dmax, s);
        if (code != BSPAI_OK) sell_free(&P, s);
        return code;
    };
    int rc;
    if ((rc = dalloc_t(&w, (size_t)S.nslices + 1, s))) return done(rc);
    if ((rc = dalloc_t(&dmax, 2, s))) return done(rc);
    if ((rc = dalloc_t(&P.sptr, (size_t)S.nslices + 1, s))) return done(rc);
    cudaError_t e = cudaMemsetAsync(dmax, 0, sizeof(unsigned), s);
    if (!e) e = cudaMemsetAsync(dmax + 1, 0x7f, sizeof(unsigned), s);
    if (e) return done(cuda_error(e, "memset", __FILE__, __LINE__));
    const unsigned grid = (unsigned)ceil_div((int64_t)S.nslices * kSlice, 256);
    if (S.nslices > 0) {
        k_packed_widths<<<grid, 256, 0, s>>>(S.n, S.nslices, S.sptr, S.col, w, dmax,
                                             reinterpret_cast<int*>(dmax + 1));
        note_launch();
        if ((e = cudaGetLastError())) return done(cuda_error(e, "k_packed_widths", __FILE__, __LINE__));
    }
    if ((rc = scan_exclusive_i64(w, P.sptr, S.nslices, s))) return done(rc);
    unsigned hd[2] = {0, 0};
    e = cudaMemcpyAsync(&P.slots, P.sptr + S.nslices, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(hd, dmax, sizeof hd, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return done(cuda_error(e, "packed sizes", __FILE__, __LINE__));
    P.maxw = S.maxw < 0 ? -1 : ((S.maxw + 3) & ~3);
    P.ellw = (S.nslices > 0 && P.maxw > 0 && (int)hd[1] == P.maxw) ? P.maxw : 0;
    if (hd[0] <= 32767u) {
        if ((rc = dalloc_t(&P.col16, (size_t)P.slots, s))) return done(rc);
    } else {
        if ((rc = dalloc_t(&P.col, (size_t)P.slots, s))) return done(rc);
    }
    float* v = nullptr;
    if ((rc = dalloc_t(&v, (size_t)P.slots, s))) return done(rc);
    if (S.nslices > 0) {
        k_packed_fill<<<grid, 256, 0, s>>>(S.n, S.nslices, S.sptr, S.col, val, P.sptr, P.col, P.col16, v);
        note_launch();
        if ((e = cudaGetLastError())) {
            dfree(v, s);
            return done(cuda_error(e, "k_packed_fill", __FILE__, __LINE__));
        }
    }
    *out = P;
    *pval = v;
    return done(BSPAI_OK);
}

__global__ void k_row_abs_sum_max(int n, const int64_t* __restrict__ sptr, const int32_t* __restrict__ col,
                                  const double* __restrict__ val, double* __restrict__ out) {
    double sum = 0.0;  // the largest row sum of this thread's rows
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = r >> 5;
        double rs = 0.0;
        for (int64_t p = sptr[s] + (r & 31); p < sptr[s + 1]; p += kSlice)
            if (col[p] >= 0) rs = __dadd_rn(rs, fabs(val[p]));
        // by bit pattern, as warp_max_bits and the atomic order them
        if ((unsigned long long)__double_as_longlong(rs) > (unsigned long long)__double_as_longlong(sum)) sum = rs;
    }
    // the max of the warp's rows, then of the block's warps: one atomic per block
    sum = warp_max_bits(sum);
    block_atomic_max_nonneg(out, sum);
}

int launch_row_abs_sum_max(const Sell& S, const double* val, double* out, cudaStream_t s) {
    if (S.n == 0) return BSPAI_OK;
    k_row_abs_sum_max<<<wave_grid(S.n), 256, 0, s>>>(S.n, S.sptr, S.col, val, out);
    note_launch();
    CUDA_LAUNCH_CHECK();
    return BSPAI_OK;
}

// ------------------------------------------------ error-free transformations
// Knuth TwoSum.
__device__ __forceinline__ void dd_two_sum(double a, double b, double& s, double& e) {
    s = __dadd_rn(a, b);
    double bv = __dsub_rn(s, a);
    e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bv)), __dsub_rn(b, bv));
}
// One term of the compensated dot product Dot2 (Ogita, Rump and Oishi, 2005):
// the running sum p absorbs -ph by TwoSum, the running error s collects the
// TwoSum error and the product's own error -pl; the result p + s is as
// accurate as a sum carried in twice the working precision (u_r ~ u^2).
__device__ __forceinline__ void dot2_sub(double& p, double& s, double ph, double pl) {
    double q;
    dd_two_sum(p, -ph, p, q);
    s = __dadd_rn(s, __dsub_rn(q, pl));
}

// r = b - A x, each product split exactly by an FMA and the terms summed by
// Dot2 in ascending column order (DD = true: u_r ~ u^2; DD = false is the
// plain fp64 recurrence), stored in the working precision (U32: rounded to
// fp32); also max|r| (of the stored r) and max|x| over rows.
template <bool DD, bool U32>
__global__ void __launch_bounds__(256) k_residual_dd(int n, const int64_t* __restrict__ sptr,
                                                     const int32_t* __restrict__ col,
                                                     const double* __restrict__ val,
                                                     const double* __restrict__ x,
                                                     const double* __restrict__ b, double* __restrict__ r,
                                                     double* __restrict__ norms) {
    double rabs = 0.0, xabs = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i >> 5;
        double hi = b[i], lo = 0.0;
        const int64_t end = sptr[s + 1];
        for (int64_t p = sptr[s] + (i & 31); p < end; p += kSlice) {
            const int c = __ldg(col + p);
            if (c < 0) break;
            const double a = __ldg(val + p);
            const double xv = __ldg(x + c);
            const double ph = __dmul_rn(a, xv);
            if (DD) {
                const double pl = __fma_rn(a, xv, -ph);
                dot2_sub(hi, lo, ph, pl);
            } else {
                hi = __dsub_rn(hi, ph);
            }
        }
        double ri = __dadd_rn(hi, lo);
        if (U32) ri = (double)__double2float_rn(ri);
        r[i] = ri;
        double ra = fabs(ri);
        if (!(ra <= 1.7976931348623157e308)) ra = __longlong_as_double(0x7ff0000000000000LL);  // NaN -> Inf
        rabs = fmax(rabs, ra);
        xabs = fmax(xabs, fabs(x[i]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rabs = fmax(rabs, __shfl_xor_sync(0xffffffffu, rabs, o));
        xabs = fmax(xabs, __shfl_xor_sync(0xffffffffu, xabs, o));
    }
    if (norms) block_atomic_max_nonneg2(norms, rabs, norms + 1, xabs);
}

// The same residual for nrhs right-hand sides of a block-diagonal batch
// (vectors stored one after another, n each; n a multiple of 32): thread per
// (right-hand side, row), and per (system, right-hand side) pair p = rhs * nsys
// + system the max |r| and max |x|, found through the system of each slice.
__global__ void __launch_bounds__(256) k_residual_batch(int n, int nrhs, const int64_t* __restrict__ sptr,
                                                        const int32_t* __restrict__ col,
                                                        const double* __restrict__ val,
                                                        const double* __restrict__ X,
                                                        const double* __restrict__ Bv, double* __restrict__ R,
                                                        const int32_t* __restrict__ slice_seg, int nsys,
                                                        double* __restrict__ prmax, double* __restrict__ pxmax) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * nrhs) return;
    const int64_t rhs = t / n;
    const int64_t i = t - rhs * n;
    const double* x = X + rhs * n;
    const int64_t s = i >> 5;
    double hi = Bv[t], lo = 0.0;
    const int64_t end = sptr[s + 1];
    for (int64_t p = sptr[s] + (i & 31); p < end; p += kSlice) {
        const int c = __ldg(col + p);
        if (c < 0) break;
        const double a = __ldg(val + p);
        const double xv = __ldg(x + c);
        const double ph = __dmul_rn(a, xv);
        const double pl = __fma_rn(a, xv, -ph);
        dot2_sub(hi, lo, ph, pl);
    }
    const double ri = __dadd_rn(hi, lo);
    R[t] = ri;
    double rabs = fabs(ri), xabs = fabs(x[i]);
    if (!(rabs <= 1.7976931348623157e308)) rabs = __longlong_as_double(0x7ff0000000000000LL);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rabs = fmax(rabs, __shfl_xor_sync(0xffffffffu, rabs, o));
        xabs = fmax(xabs, __shfl_xor_sync(0xffffffffu, xabs, o));
    }
    if ((threadIdx.x & 31) == 0) {
        const int64_t pair = rhs * nsys + slice_seg[s];
        atomic_max_nonneg(prmax + pair, rabs);
        atomic_max_nonneg(pxmax + pair, xabs);
    }
}

int launch_residual_batch(const bspai_matrix* A, int nrhs, const double* X, const double* Bv, double* R,
                          const int32_t* slice_seg, int nsys, double* prmax, double* pxmax, cudaStream_t s) {
    const int64_t total = (int64_t)A->n * nrhs;
    if (total == 0) return BSPAI_OK;
    ProfScope ps(BSPAI_K_RESIDUAL, s);
    k_residual_batch<<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(A->n, nrhs, A->sell.sptr, A->sell.col, A->val64,
                                                                    X, Bv, R, slice_seg, nsys, prmax, pxmax);
    note_launch();
    CUDA_LAUNCH_CHECK();
    return BSPAI_OK;
}

int launch_residual_prec(const bspai_matrix* A, const double* x, const double* b, double* r, double* norms,
                         int u_r, int u, cudaStream_t s) {
    if (A->n == 0) return BSPAI_OK;
    ProfScope ps(BSPAI_K_RESIDUAL, s);
    const unsigned grid = wave_grid(A->n);
    const int64_t* sp = A->sell.sptr;
    const int32_t* ci = A->sell.col;
    if (u == BSPAI_FP32) {
        if (u_r == BSPAI_FP64)
            k_residual_dd<false, true><<<grid, 256, 0, s>>>(A->n, sp, ci, A->val64, x, b, r, norms);
        else
            k_residual_dd<true, true><<<grid, 256, 0, s>>>(A->n, sp, ci, A->val64, x, b, r, norms);
    } else {
        if (u_r == BSPAI_FP64)
            k_residual_dd<false, false><<<grid, 256, 0, s>>>(A->n, sp, ci, A->val64, x, b, r, norms);
        else
            k_residual_dd<true, false><<<grid, 256, 0, s>>>(A->n, sp, ci, A->val64, x, b, r, norms);
    }
    note_launch();
    CUDA_LAUNCH_CHECK();
    return BSPAI_OK;
}

int launch_residual(const bspai_matrix* A, const double* x, const double* b, double* r, double* norms,
                    cudaStream_t s) {
    return launch_residual_prec(A, x, b, r, norms, BSPAI_DD, BSPAI_FP64, s);
}

// Structural check of a caller CSR before any kernel indexes through it:
// row_ptr[0] = 0, row_ptr[n] = nnz, non-decreasing, columns in [0, n) and
// strictly ascending within each row.  Bit 0: bad row pointers, bit 1: bad
// column, bit 2: unsorted or repeated column.
__global__ void k_validate_csr(int n, int nnz, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                               int* __restrict__ bad) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n) return;
    if (r == n) {
        if (rp[n] != nnz || rp[0] != 0) atomicOr(bad, 1);
        return;
    }
    const int b = rp[r], e = rp[r + 1];
    if (b < 0 || e < b || e > nnz) {
        atomicOr(bad, 1);
        return;
    }
    if (!col) return;
    for (int p = b; p < e; ++p) {
        const int c = col[p];
        if (c < 0 || c >= n) atomicOr(bad, 2);
        else if (p > b && c <= col[p - 1]) atomicOr(bad, 4);
    }
}

int validate_csr(const bspai_csr_t* A, bool need_val, const char* who, cudaStream_t s) {
    if (!A) return set_error(BSPAI_ERR_INVALID, "%s: null matrix", who);
    if (A->n < 0 || A->nnz < 0) return set_error(BSPAI_ERR_INVALID, "%s: negative size", who);
    if (A->n == 0) return BSPAI_OK;
    if (!A->row_ptr || (A->nnz > 0 && !A->col) || (need_val && A->nnz > 0 && !A->val))
        return set_error(BSPAI_ERR_INVALID, "%s: missing CSR arrays", who);
    int* d_bad = nullptr;
    BSPAI_TRY(dalloc_t(&d_bad, 1, s));
    CUDA_TRY(cudaMemsetAsync(d_bad, 0, sizeof(int), s));
    k_validate_csr<<<(unsigned)ceil_div((int64_t)A->n + 1, 256), 256, 0, s>>>(A->n, A->nnz, A->row_ptr, A->col,
                                                                              d_bad);
    note_launch();
    CUDA_LAUNCH_CHECK();
    int bad = 0;
    CUDA_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    dfree(d_bad, s);
    if (bad)
        return set_error(BSPAI_ERR_INVALID, "%s: malformed CSR (%s%s%s)", who, (bad & 1) ? "row pointers " : "",
                         (bad & 2) ? "column out of range " : "", (bad & 4) ? "columns not strictly ascending" : "");
    return BSPAI_OK;
}

int matrix_create(const bspai_csr_t* A, cudaStream_t s, bspai_matrix** out) {
    if (!A || !out) return set_error(BSPAI_ERR_INVALID, "matrix_create: null argument");
    if (A->n < 0 || A->nnz < 0) return set_error(BSPAI_ERR_INVALID, "matrix_create: negative size");
    if (A->n > 0 && (!A->row_ptr || !A->col || !A->val))
        return set_error(BSPAI_ERR_INVALID, "matrix_create: A needs row_ptr, col and val");
    BSPAI_TRY(validate_csr(A, true, "matrix_create", s));
    auto* M = new bspai_matrix();
    M->magic = kMagicA;
    M->stream = s;
    M->n = A->n;
    M->nnz = A->nnz;
    int st;
    {
        ProfScope ps(BSPAI_K_OTHER, s);
        st = sell_from_csr(A->n, A->row_ptr, A->col, A->val, &M->sell, &M->val64, &M->val32, &M->rowlen, s);
        if (st == BSPAI_OK) st = dalloc_t(&M->csr_row_ptr, (size_t)A->n + 1, s);
        if (st == BSPAI_OK) {
            cudaError_t e = cudaMemcpyAsync(M->csr_row_ptr, A->row_ptr, sizeof(int32_t) * ((size_t)A->n + 1),
                                            cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) st = cuda_error(e, "copy", __FILE__, __LINE__);
        }
        if (st == BSPAI_OK) st = dalloc_t(&M->norm_inf, 1, s);
        if (st == BSPAI_OK) {
            cudaError_t e = cudaMemsetAsync(M->norm_inf, 0, sizeof(double), s);
            if (e != cudaSuccess) st = cuda_error(e, "memset", __FILE__, __LINE__);
        }
        if (st == BSPAI_OK && A->n > 0) {
            k_row_abs_sum_max<<<wave_grid(A->n), 256, 0, s>>>(A->n, M->sell.sptr, M->sell.col,
                                                                            M->val64, M->norm_inf);
            note_launch();
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) st = cuda_error(e, "k_row_abs_sum_max", __FILE__, __LINE__);
        }
        if (st == BSPAI_OK) st = sell_packed_copy(M->sell, M->val32, &M->psell, &M->pval32, s);
    }
    if (st != BSPAI_OK) {
        bspai_free(M);
        return st;
    }
    *out = M;
    return BSPAI_OK;
}

}  // namespace bspai

using namespace bspai;

extern "C" {

int bspai_matrix_create(const bspai_csr_t* A, bspai_stream_t s, bspai_A_h* out) {
    if (!out) return set_error(BSPAI_ERR_INVALID, "bspai_matrix_create: null out");
    *out = nullptr;
    return matrix_create(A, (cudaStream_t)s, out);
}

int bspai_residual(bspai_A_h A, const double* x, const double* b, double* r, bspai_stream_t s) {
    if (!A || A->magic != kMagicA) return set_error(BSPAI_ERR_INVALID, "bspai_residual: bad handle");
    if (A->n > 0 && (!x || !b || !r)) return set_error(BSPAI_ERR_INVALID, "bspai_residual: null vector");
    return launch_residual(A, x, b, r, nullptr, (cudaStream_t)s);
}

int bspai_residual_prec(bspai_A_h A, const double* x, const double* b, bspai_prec_t u_r, bspai_prec_t u, double* r,
                        bspai_stream_t s) {
    if (!A || A->magic != kMagicA) return set_error(BSPAI_ERR_INVALID, "bspai_residual_prec: bad handle");
    if (u_r != BSPAI_DD && u_r != BSPAI_FP64)
        return set_error(BSPAI_ERR_UNSUPPORTED, "bspai_residual_prec: u_r must be DD or FP64");
    if (u != BSPAI_FP64 && u != BSPAI_FP32)
        return set_error(BSPAI_ERR_UNSUPPORTED, "bspai_residual_prec: u must be FP64 or FP32");
    if (A->n > 0 && (!x || !b || !r)) return set_error(BSPAI_ERR_INVALID, "bspai_residual_prec: null vector");
    return launch_residual_prec(A, x, b, r, nullptr, u_r, u, (cudaStream_t)s);
}

}  // extern "C"
