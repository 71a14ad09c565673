// transpose.cu -- transposed operators for the adjoint solve A^T lambda = g,
// left-preconditioned by the transpose of the bucketed M (the same buckets and
// stored values, read by rows of M^T), and the gradient dL/dA_ij = -lambda_i x_j
// on the nonzeros of A.
//
// Any SELL-32 matrix is transposed in four steps: count the entries of every
// column, scan, scatter (row index, source slot) into CSR rows of the
// transpose, sort each row by column (short rows: insertion sort, one thread
// per row); then the CSR structure is packed into SELL-32 and each value is
// copied from its source slot.  The payload is moved byte for byte, so the
// transposed operator stores exactly the same values.
#include "common.cuh"

namespace bspai {

int launch_row_abs_sum_max(const Sell& S, const double* val, double* out, cudaStream_t s);

// (both read the source in either slot arrangement and either index width)
__global__ void k_tcount(int n, const int64_t* __restrict__ sptr, const int32_t* __restrict__ col,
                         const int16_t* __restrict__ col16, int packed, unsigned long long* __restrict__ cnt) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t b = sptr[r >> 5];
    const int w = (int)((sptr[(r >> 5) + 1] - b) >> 5);
    for (int l = 0; l < w; ++l) {
        const int c = sell_col(col, col16, sell_slot(b, (int)(r & 31), l, packed), r);
        if (c >= 0) atomicAdd(cnt + c, 1ull);
    }
}

__global__ void k_i64_to_i32(int64_t count, const int64_t* __restrict__ in, int32_t* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = (int32_t)in[i];
}

__global__ void k_tscatter(int n, const int64_t* __restrict__ sptr, const int32_t* __restrict__ col,
                           const int16_t* __restrict__ col16, int packed, const int32_t* __restrict__ trp,
                           unsigned* __restrict__ cur, int32_t* __restrict__ tcol, int64_t* __restrict__ tsrc) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t b = sptr[r >> 5];
    const int w = (int)((sptr[(r >> 5) + 1] - b) >> 5);
    for (int l = 0; l < w; ++l) {
        const int64_t p = sell_slot(b, (int)(r & 31), l, packed);
        const int c = sell_col(col, col16, p, r);
        if (c < 0) continue;
        const int64_t pos = trp[c] + atomicAdd(cur + c, 1u);
        tcol[pos] = (int32_t)r;
        tsrc[pos] = p;
    }
}

__global__ void k_tsort(int n, const int32_t* __restrict__ trp, int32_t* __restrict__ tcol, int64_t* __restrict__ tsrc) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int b = trp[c], e = trp[c + 1];
    for (int i = b + 1; i < e; ++i) {
        const int32_t k = tcol[i];
        const int64_t v = tsrc[i];
        int j = i - 1;
        while (j >= b && tcol[j] > k) {
            tcol[j + 1] = tcol[j];
            tsrc[j + 1] = tsrc[j];
            --j;
        }
        tcol[j + 1] = k;
        tsrc[j + 1] = v;
    }
}

// copy the payload (esize bytes per entry) from source slots to the slots of the transpose
__global__ void k_tgather(int n, const int64_t* __restrict__ tsptr, const int32_t* __restrict__ trowlen,
                          const int32_t* __restrict__ trp, const int64_t* __restrict__ tsrc, int esize,
                          const unsigned char* __restrict__ src, unsigned char* __restrict__ dst) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t b = tsptr[r >> 5] + (r & 31);
    const int len = trowlen[r];
    for (int l = 0; l < len; ++l) {
        const int64_t s = tsrc[trp[r] + l];
        const int64_t d = b + (int64_t)l * kSlice;
        switch (esize) {
        case 8: reinterpret_cast<uint64_t*>(dst)[d] = reinterpret_cast<const uint64_t*>(src)[s]; break;
        case 4: reinterpret_cast<uint32_t*>(dst)[d] = reinterpret_cast<const uint32_t*>(src)[s]; break;
        case 2: reinterpret_cast<uint16_t*>(dst)[d] = reinterpret_cast<const uint16_t*>(src)[s]; break;
        default: dst[d] = src[s]; break;
        }
    }
}

// Structure of S^T as CSR (row pointers int32, columns ascending) plus, per
// entry, the slot of S it came from; then packed into SELL-32.
struct TransposeMap {
    int32_t* trp = nullptr;
    int32_t* tcol = nullptr;
    int64_t* tsrc = nullptr;
    void release(cudaStream_t s) {
        dfree(trp, s);
        dfree(tcol, s);
        dfree(tsrc, s);
    }
};

static int transpose_structure(const Sell& S, int64_t nnz, TransposeMap& T, Sell* out, int32_t** rowlen,
                               cudaStream_t s) {
    const int n = S.n;
    unsigned long long* cnt = nullptr;
    int64_t* rp64 = nullptr;
    unsigned* cur = nullptr;
    auto done = [&](int code) {
        dfree(cnt, s);
        dfree(rp64, s);
        dfree(cur, s);
        return code;
    };
    int rc;
    if ((rc = dalloc_t(&cnt, (size_t)n + 1, s))) return done(rc);
    if ((rc = dalloc_t(&rp64, (size_t)n + 1, s))) return done(rc);
    if ((rc = dalloc_t(&cur, (size_t)n + 1, s))) return done(rc);
    if ((rc = dalloc_t(&T.trp, (size_t)n + 1, s))) return done(rc);
    if ((rc = dalloc_t(&T.tcol, (size_t)(nnz > 0 ? nnz : 1), s))) return done(rc);
    if ((rc = dalloc_t(&T.tsrc, (size_t)(nnz > 0 ? nnz : 1), s))) return done(rc);
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * ((size_t)n + 1), s);
    if (!e) e = cudaMemsetAsync(cur, 0, sizeof(unsigned) * ((size_t)n + 1), s);
    if (e) return done(cuda_error(e, "transpose setup", __FILE__, __LINE__));
    const unsigned g = (unsigned)ceil_div(n, 256);
    if (n > 0) {
        k_tcount<<<g, 256, 0, s>>>(n, S.sptr, S.col, S.col16, S.packed, cnt);
        note_launch();
    }
    if ((rc = scan_exclusive_i64(reinterpret_cast<const int64_t*>(cnt), rp64, n, s))) return done(rc);
    k_i64_to_i32<<<(unsigned)ceil_div((int64_t)n + 1, 256), 256, 0, s>>>((int64_t)n + 1, rp64, T.trp);
    note_launch();
    if (n > 0) {
        k_tscatter<<<g, 256, 0, s>>>(n, S.sptr, S.col, S.col16, S.packed, T.trp, cur, T.tcol, T.tsrc);
        note_launch();
        k_tsort<<<g, 256, 0, s>>>(n, T.trp, T.tcol, T.tsrc);
        note_launch();
    }
    if ((e = cudaGetLastError())) return done(cuda_error(e, "transpose kernels", __FILE__, __LINE__));
    if ((rc = sell_from_csr(n, T.trp, T.tcol, nullptr, out, nullptr, nullptr, rowlen, s))) return done(rc);
    return done(BSPAI_OK);
}

static int gather_payload(const Sell& St, const int32_t* rowlen, const TransposeMap& T, int esize, const void* src,
                          void** dst, cudaStream_t s) {
    BSPAI_TRY(dalloc(dst, (size_t)St.slots * esize, s));
    CUDA_TRY(cudaMemsetAsync(*dst, 0, (size_t)St.slots * esize, s));
    if (St.n > 0) {
        k_tgather<<<(unsigned)ceil_div(St.n, 256), 256, 0, s>>>(St.n, St.sptr, rowlen, T.trp, T.tsrc, esize,
                                                                (const unsigned char*)src, (unsigned char*)*dst);
        note_launch();
        CUDA_LAUNCH_CHECK();
    }
    return BSPAI_OK;
}

static size_t prec_size(int prec) {
    switch (prec) {
    case BSPAI_FP64: return 8;
    case BSPAI_FP32: return 4;
    case BSPAI_FP16:
    case BSPAI_BF16: return 2;
    case BSPAI_E4M3: return 1;
    default: return 0;
    }
}

// dA[p] = sum_r -lambda_r[i] x_r[j] over the nrhs right-hand sides (r ascending,
// fp64, each product and sum rounded once), for the p-th nonzero (i, j) of A
__global__ void k_adjoint_grad(int n, int nrhs, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                               const double* __restrict__ lambda, const double* __restrict__ x,
                               double* __restrict__ dA) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p0 = rp[i], p1 = rp[i + 1];
    for (int p = p0; p < p1; ++p) {
        const int64_t c = col[p];
        double acc = 0.0;
        for (int r = 0; r < nrhs; ++r)
            acc = __dadd_rn(acc, __dmul_rn(-lambda[(int64_t)r * n + i], x[(int64_t)r * n + c]));
        dA[p] = acc;
    }
}

}  // namespace bspai

using namespace bspai;

extern "C" {

int bspai_matrix_transpose(bspai_A_h A, bspai_stream_t st, bspai_A_h* out) {
    cudaStream_t s = (cudaStream_t)st;
    if (!out) return set_error(BSPAI_ERR_INVALID, "bspai_matrix_transpose: null out");
    *out = nullptr;
    if (!A || A->magic != kMagicA) return set_error(BSPAI_ERR_INVALID, "bspai_matrix_transpose: bad handle");
    auto* T = new bspai_matrix();
    T->magic = kMagicA;
    T->stream = s;
    T->n = A->n;
    T->nnz = A->nnz;
    TransposeMap map;
    int32_t* rowlen = nullptr;
    int rc = BSPAI_OK;
    {
        ProfScope ps(BSPAI_K_OTHER, s);
        rc = transpose_structure(A->sell, A->nnz, map, &T->sell, &rowlen, s);
        void* p = nullptr;
        if (!rc) rc = gather_payload(T->sell, rowlen, map, 8, A->val64, &p, s);
        T->val64 = (double*)p;
        p = nullptr;
        if (!rc) rc = gather_payload(T->sell, rowlen, map, 4, A->val32, &p, s);
        T->val32 = (float*)p;
        if (!rc) rc = sell_packed_copy(T->sell, T->val32, &T->psell, &T->pval32, s);
        if (!rc) rc = dalloc_t(&T->norm_inf, 1, s);
        if (!rc) {
            cudaError_t e = cudaMemsetAsync(T->norm_inf, 0, sizeof(double), s);
            if (e) rc = cuda_error(e, "memset", __FILE__, __LINE__);
        }
        if (!rc) rc = launch_row_abs_sum_max(T->sell, T->val64, T->norm_inf, s);
    }
    map.release(s);
    dfree(rowlen, s);
    if (rc) {
        bspai_free(T);
        return rc;
    }
    *out = T;
    return BSPAI_OK;
}

int bspai_M_transpose(bspai_M_h M, bspai_stream_t st, bspai_M_h* out) {
    cudaStream_t s = (cudaStream_t)st;
    if (!out) return set_error(BSPAI_ERR_INVALID, "bspai_M_transpose: null out");
    *out = nullptr;
    if (!M || M->magic != kMagicM) return set_error(BSPAI_ERR_INVALID, "bspai_M_transpose: bad handle");
    auto* T = new bspai_spai();
    T->magic = kMagicM;
    T->stream = s;
    T->n = M->n;
    T->nnz = M->nnz;
    T->uf = M->uf;
    TransposeMap map;
    int rc = BSPAI_OK;
    {
        ProfScope ps(BSPAI_K_OTHER, s);
        rc = transpose_structure(M->sell, M->nnz, map, &T->sell, &T->rowlen, s);
        void* p = nullptr;
        if (!rc) rc = gather_payload(T->sell, T->rowlen, map, 4, M->val, &p, s);
        T->val = (float*)p;
        if (!rc) rc = dalloc_t(&T->csr_row_ptr, (size_t)T->n + 1, s);
        if (!rc) {
            cudaError_t e = cudaMemcpyAsync(T->csr_row_ptr, map.trp, sizeof(int32_t) * ((size_t)T->n + 1),
                                            cudaMemcpyDeviceToDevice, s);
            if (e) rc = cuda_error(e, "copy", __FILE__, __LINE__);
        }
        if (!rc) rc = dalloc_t(&T->resid, (size_t)(T->n > 0 ? T->n : 1), s);
        if (!rc) {
            // column residuals belong to M, not to its transpose
            cudaError_t e = cudaMemsetAsync(T->resid, 0, sizeof(float) * (size_t)(T->n > 0 ? T->n : 1), s);
            if (e) rc = cuda_error(e, "memset", __FILE__, __LINE__);
        }
    }
    map.release(s);
    if (rc) {
        bspai_free(T);
        return rc;
    }
    *out = T;
    return BSPAI_OK;
}

int bspai_bucket_transpose(bspai_BM_h BM, bspai_stream_t st, bspai_BM_h* out) {
    cudaStream_t s = (cudaStream_t)st;
    if (!out) return set_error(BSPAI_ERR_INVALID, "bspai_bucket_transpose: null out");
    *out = nullptr;
    if (!BM || BM->magic != kMagicBM) return set_error(BSPAI_ERR_INVALID, "bspai_bucket_transpose: bad handle");
    if (BM->rowscale) return set_error(BSPAI_ERR_UNSUPPORTED, "bspai_bucket_transpose: already a transpose");
    auto* T = new bspai_bucketed();
    T->magic = kMagicBM;
    T->stream = s;
    T->n = BM->n;
    T->nnz = BM->nnz;
    T->q = BM->q;
    int rc = BSPAI_OK;
    {
        ProfScope ps(BSPAI_K_OTHER, s);
        for (int k = 0; k < BM->q && !rc; ++k) {
            T->precs[k] = BM->precs[k];
            T->scale[k] = BM->scale[k];
            T->nnz_k[k] = BM->nnz_k[k];
            T->maxw[k] = -1;
            const size_t es = prec_size(BM->precs[k]);
            if (es == 0) {  // dropped: nothing stored, keep an empty structure
                T->b[k].n = BM->n;
                T->b[k].nslices = BM->b[k].nslices;
                T->b[k].slots = 0;
                rc = dalloc_t(&T->b[k].sptr, (size_t)T->b[k].nslices + 1, s);
                if (!rc) {
                    cudaError_t e = cudaMemsetAsync(T->b[k].sptr, 0, sizeof(int64_t) * ((size_t)T->b[k].nslices + 1), s);
                    if (e) rc = cuda_error(e, "memset", __FILE__, __LINE__);
                }
                continue;
            }
            TransposeMap map;
            int32_t* rowlen = nullptr;
            rc = transpose_structure(BM->b[k], BM->nnz_k[k], map, &T->b[k], &rowlen, s);
            if (!rc && BM->sscale[k]) {
                // block-diagonal batch: the slices of M^T cover the same systems
                rc = dalloc_t(&T->sscale[k], (size_t)BM->b[k].nslices, s);
                if (!rc) {
                    cudaError_t e = cudaMemcpyAsync(T->sscale[k], BM->sscale[k], sizeof(float) * BM->b[k].nslices,
                                                    cudaMemcpyDeviceToDevice, s);
                    if (e) rc = cuda_error(e, "copy", __FILE__, __LINE__);
                }
            }
            if (!rc) rc = gather_payload(T->b[k], rowlen, map, (int)es, BM->val[k], &T->val[k], s);
            if (!rc) T->maxw[k] = T->b[k].maxw;
            map.release(s);
            dfree(rowlen, s);
        }
        if (!rc && BM->colscale) {
            // the per-column scale of an e4m3 bucket of M is a per-row scale of M^T
            rc = dalloc_t(&T->rowscale, (size_t)BM->n, s);
            if (!rc) {
                cudaError_t e = cudaMemcpyAsync(T->rowscale, BM->colscale, sizeof(float) * (size_t)BM->n,
                                                cudaMemcpyDeviceToDevice, s);
                if (e) rc = cuda_error(e, "copy", __FILE__, __LINE__);
            }
        }
    }
    if (rc) {
        bspai_free(T);
        return rc;
    }
    *out = T;
    return BSPAI_OK;
}

int bspai_adjoint_grad_A(const bspai_csr_t* A, int32_t nrhs, const double* lambda, const double* x, double* dA,
                         bspai_stream_t st) {
    cudaStream_t s = (cudaStream_t)st;
    if (!A || A->n < 0) return set_error(BSPAI_ERR_INVALID, "bspai_adjoint_grad_A: bad matrix");
    if (nrhs < 1) return set_error(BSPAI_ERR_INVALID, "bspai_adjoint_grad_A: nrhs = %d", nrhs);
    if (A->n == 0) return BSPAI_OK;
    if (!A->row_ptr || !A->col || !lambda || !x || !dA)
        return set_error(BSPAI_ERR_INVALID, "bspai_adjoint_grad_A: null pointer");
    ProfScope ps(BSPAI_K_OTHER, s);
    k_adjoint_grad<<<(unsigned)ceil_div(A->n, 256), 256, 0, s>>>(A->n, nrhs, A->row_ptr, A->col, lambda, x, dA);
    note_launch();
    CUDA_LAUNCH_CHECK();
    return BSPAI_OK;
}

}  // extern "C"
