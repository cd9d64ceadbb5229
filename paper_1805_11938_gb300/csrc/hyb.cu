// HYB = ELL + COO (Sec. II-B "HYB"): the first K entries of every row go to a
// column-major ELL, the rest to a COO tail.  K is the "typical" row length:
// the largest k such that at least ceil(m/3) rows hold k or more entries.
//
// The tail is kept grouped by row (tail_rows, tail_ptr: COO sorted by row,
// CSR order inside a row), so it is summed without atomics: the ELL kernel
// writes every y_i, then the CSR tile kernel adds each tail row's sum to
// its own y_i (one writer per row, stream-ordered after the ELL part).
#include "internal.cuh"
#include "kernels.cuh"

namespace spmv {

using dev::row_of_nnz;

__global__ void k_len_hist(const int32_t* __restrict__ len, int32_t m, int32_t* __restrict__ hist) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) atomicAdd(hist + len[i], 1);
}

// rev[b] = hist[maxlen - b]
__global__ void k_reverse(const int32_t* __restrict__ hist, int32_t maxlen, int32_t* __restrict__ rev) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b <= maxlen) rev[b] = hist[maxlen - b];
}

// K = #{k in [1, maxlen] : c_k >= need}, c_k = rows with length >= k = E[maxlen - k + 1]
__global__ void k_count_k(const int32_t* __restrict__ E, int32_t maxlen, int32_t need, int32_t* __restrict__ K) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x + 1;
    int ok = (k <= maxlen) && (E[maxlen - k + 1] >= need);
    ok = __syncthreads_count(ok);
    if (threadIdx.x == 0 && ok) atomicAdd(K, ok);
}

__global__ void k_tail_flags(const int32_t* __restrict__ len, int32_t m, int32_t K, int32_t* __restrict__ has,
                             int32_t* __restrict__ tl) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i <= m) {
        const int32_t t = (i < m && len[i] > K) ? len[i] - K : 0;
        has[i] = t > 0;
        tl[i] = t;
    }
}

__global__ void k_tail_rows(const int32_t* __restrict__ has, const int32_t* __restrict__ tpos,
                            const int32_t* __restrict__ tl, int32_t m, int32_t* __restrict__ rows,
                            int32_t* __restrict__ tlen) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m && has[i]) {
        rows[tpos[i]] = (int32_t)i;
        tlen[tpos[i]] = tl[i];
    }
}

__global__ void k_tail_scatter(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                               const double* __restrict__ val, int32_t m, int64_t nnz, int32_t K,
                               const int32_t* __restrict__ tpos, const int32_t* __restrict__ tptr,
                               int32_t* __restrict__ tcol, double* __restrict__ tval) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = row_of_nnz(ptr, m, k);
        const int64_t j = k - ptr[r];
        if (j >= K) {
            const int64_t d = tptr[tpos[r]] + (j - K);
            tcol[d] = idx[k];
            tval[d] = val[k];
        }
    }
}

int hyb_convert(spmv_handle* h, const spmv_csr* c, cudaStream_t s) {
    const int32_t m = c->m;
    Scratch tmp;
    int32_t* len = nullptr;
    SPMV_TRY(tmp.get(&len, (size_t)m + 1));
    SPMV_TRY(row_lengths(c->ptr, m, len, s));
    int32_t maxlen = 0;
    SPMV_TRY(max_i32(len, m, &maxlen, s, tmp));
    int32_t K = 0;
    if (h->params.hyb_k > 0) {
        K = h->params.hyb_k < maxlen ? h->params.hyb_k : maxlen;
    } else if (h->params.hyb_k == 0) {
        int32_t *hist = nullptr, *rev = nullptr, *E = nullptr, *dK = nullptr;
        SPMV_TRY(tmp.get(&hist, (size_t)maxlen + 1));
        SPMV_TRY(tmp.get(&rev, (size_t)maxlen + 1));
        SPMV_TRY(tmp.get(&E, (size_t)maxlen + 2));
        SPMV_TRY(tmp.get(&dK, 1));
        SPMV_CUDA(cudaMemsetAsync(hist, 0, sizeof(int32_t) * ((size_t)maxlen + 1), s));
        SPMV_CUDA(cudaMemsetAsync(dK, 0, sizeof(int32_t), s));
        k_len_hist<<<grid_for(m, 256), 256, 0, s>>>(len, m, hist);
        k_reverse<<<grid_for((int64_t)maxlen + 1, 256), 256, 0, s>>>(hist, maxlen, rev);
        SPMV_CUDA(cudaGetLastError());
        SPMV_TRY(exclusive_scan<int32_t>(rev, E, (int64_t)maxlen + 1, s, tmp));
        const int32_t need = (int32_t)(((int64_t)m + 2) / 3);
        if (maxlen > 0) k_count_k<<<grid_for(maxlen, 256), 256, 0, s>>>(E, maxlen, need, dK);
        SPMV_CUDA(cudaGetLastError());
        SPMV_CUDA(cudaMemcpyAsync(&K, dK, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SPMV_CUDA(cudaStreamSynchronize(s));
    } else if (h->params.hyb_k != SPMV_HYB_K_NONE) {
        return set_error(SPMV_ERR_INVALID_ARG, "hyb_k must be > 0, 0 (rule) or SPMV_HYB_K_NONE (got %d)", h->params.hyb_k);
    }
    h->params.hyb_k = K;
    SPMV_TRY(ell_build(h, h->ell, c, K, len, true, s));
    // tail rows and their entries
    int32_t *has = nullptr, *tl = nullptr, *tpos = nullptr, *tlen = nullptr;
    SPMV_TRY(tmp.get(&has, (size_t)m + 1));
    SPMV_TRY(tmp.get(&tl, (size_t)m + 1));
    SPMV_TRY(tmp.get(&tpos, (size_t)m + 2));
    k_tail_flags<<<grid_for((int64_t)m + 1, 256), 256, 0, s>>>(len, m, K, has, tl);
    SPMV_CUDA(cudaGetLastError());
    SPMV_TRY(exclusive_scan<int32_t>(has, tpos, (int64_t)m + 1, s, tmp));
    int32_t ntr = 0;
    SPMV_CUDA(cudaMemcpyAsync(&ntr, tpos + m, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA(cudaStreamSynchronize(s));
    h->n_tail_rows = ntr;
    SPMV_TRY(tmp.get(&tlen, (size_t)ntr + 1));
    SPMV_TRY(h->alloc(&h->tail_rows, (size_t)ntr + 1, "tail_rows"));
    SPMV_TRY(h->alloc(&h->tail_ptr, (size_t)ntr + 1, "tail_ptr"));
    k_tail_rows<<<grid_for(m, 256), 256, 0, s>>>(has, tpos, tl, m, h->tail_rows, tlen);
    SPMV_CUDA(cudaGetLastError());
    SPMV_TRY(exclusive_scan<int32_t>(tlen, h->tail_ptr, ntr, s, tmp));
    int32_t nt = 0;
    SPMV_CUDA(cudaMemcpyAsync(&nt, h->tail_ptr + ntr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA(cudaStreamSynchronize(s));
    h->n_tail = nt;
    SPMV_TRY(h->alloc(&h->tail_col, (size_t)nt, "tail_col"));
    SPMV_TRY(h->alloc(&h->tail_val, (size_t)nt, "tail_val"));
    if (nt > 0) {
        int g = grid_capped(c->nnz, 256, 64);
        k_tail_scatter<<<g, 256, 0, s>>>(c->ptr, c->idx, c->val, m, c->nnz, K, tpos, h->tail_ptr, h->tail_col,
                                         h->tail_val);
        SPMV_CUDA(cudaGetLastError());
    }
    SPMV_TRY(build_csr_tiles(h, h->tail_units, h->tail_ptr, ntr, nt, "tail_", s));
    SPMV_TRY(csr_prepare(h->tail_units));
    h->stored_slots += nt;
    h->aux[0] = nt;
    h->aux[1] = ntr;
    h->aux[2] = K;
    h->aux[3] = h->tail_units.n;
    return SPMV_OK;
}

int hyb_run(const spmv_handle* h, const double* x, double* y, cudaStream_t s) {
    SPMV_TRY(ell_launch(h->ell, h->m, 0x7fffffff, x, y, s));
    if (h->n_tail_rows > 0)
        SPMV_TRY(csr_tiles_launch(h->tail_units, h->tail_ptr, h->tail_col, h->tail_val, h->tail_rows, x, y, true, s));
    return SPMV_OK;
}

__global__ void k_hyb_len(const int32_t* __restrict__ row_len, int32_t m, int32_t* __restrict__ len,
                          int32_t* __restrict__ tpos) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) {
        len[i] = row_len[i];
        tpos[i] = -1;
    }
}

__global__ void k_hyb_tail_len(const int32_t* __restrict__ rows, const int32_t* __restrict__ tptr, int32_t ntr,
                               int32_t* __restrict__ len, int32_t* __restrict__ tpos) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < ntr) {
        len[rows[t]] += tptr[t + 1] - tptr[t];
        tpos[rows[t]] = (int32_t)t;
    }
}

__global__ void k_hyb_gather(const int32_t* __restrict__ ptr, int32_t m, int64_t nnz, int32_t K, int64_t ld,
                             const int32_t* __restrict__ col, const double* __restrict__ ev,
                             const int32_t* __restrict__ tpos, const int32_t* __restrict__ tptr,
                             const int32_t* __restrict__ tcol, const double* __restrict__ tval,
                             int32_t* __restrict__ idx, double* __restrict__ val) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = row_of_nnz(ptr, m, k);
        const int64_t j = k - ptr[r];
        if (j < K) {
            idx[k] = col[j * ld + r];
            val[k] = ev[j * ld + r];
        } else {
            const int64_t d = tptr[tpos[r]] + (j - K);
            idx[k] = tcol[d];
            val[k] = tval[d];
        }
    }
}

int hyb_to_csr(const spmv_handle* h, int32_t* ptr, int32_t* idx, double* val, cudaStream_t s) {
    Scratch tmp;
    int32_t *len = nullptr, *tpos = nullptr;
    SPMV_TRY(tmp.get(&len, (size_t)h->m));
    SPMV_TRY(tmp.get(&tpos, (size_t)h->m));
    k_hyb_len<<<grid_for(h->m, 256), 256, 0, s>>>(h->ell.row_len, h->m, len, tpos);
    if (h->n_tail_rows > 0)
        k_hyb_tail_len<<<grid_for(h->n_tail_rows, 256), 256, 0, s>>>(h->tail_rows, h->tail_ptr, h->n_tail_rows, len,
                                                                      tpos);
    SPMV_CUDA(cudaGetLastError());
    SPMV_TRY(exclusive_scan<int32_t>(len, ptr, h->m, s, tmp));
    if (h->nnz > 0) {
        int g = grid_capped(h->nnz, 256, 64);
        k_hyb_gather<<<g, 256, 0, s>>>(ptr, h->m, h->nnz, h->ell.K, h->ell.ld, h->ell.col, h->ell.val, tpos,
                                       h->tail_ptr, h->tail_col, h->tail_val, idx, val);
    }
    SPMV_CUDA(cudaGetLastError());
    SPMV_CUDA(cudaStreamSynchronize(s));
    return SPMV_OK;
}

}  // namespace spmv
