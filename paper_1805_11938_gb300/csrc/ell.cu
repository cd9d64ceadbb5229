// ELL (Sec. II-B "ELL"): K = the longest row; every row padded to K slots.
// Stored column-major (slot s of row i at s*ld + i, ld = m rounded up to a
// multiple of 4) so that consecutive rows are consecutive in memory; padding
// holds column 0 and value +0.0 and is never multiplied (row_len bounds every
// loop).  The same layout is the ELL part of HYB.
#include "internal.cuh"
#include "kernels.cuh"

namespace spmv {

using dev::row_of_nnz;

__global__ void k_ell_row_len(const int32_t* __restrict__ len, int32_t m, int32_t K, int32_t* __restrict__ row_len) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) row_len[i] = len[i] < K ? len[i] : K;
}

__global__ void k_ell_scatter(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                              const double* __restrict__ val, int32_t m, int64_t nnz, int32_t K, int64_t ld,
                              int32_t* __restrict__ col, double* __restrict__ ev) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = row_of_nnz(ptr, m, k);
        const int64_t j = k - ptr[r];
        if (j < K) {
            col[j * ld + r] = idx[k];
            ev[j * ld + r] = val[k];
        }
    }
}

__global__ void k_flag_long(const int32_t* __restrict__ row_len, int32_t m, int32_t long_len, int32_t* __restrict__ f) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i <= m) f[i] = (i < m && row_len[i] > long_len) ? 1 : 0;
}

__global__ void k_compact(const int32_t* __restrict__ f, const int32_t* __restrict__ off, int32_t m,
                          int32_t* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m && f[i]) out[off[i]] = (int32_t)i;
}

int ell_build(spmv_handle* h, EllPart& e, const spmv_csr* c, int32_t K, const int32_t* len, bool hyb,
              cudaStream_t s) {
    const int32_t m = c->m;
    e.K = K;
    e.ld = ceil_div(m, 4) * 4;
    const int64_t slots = (int64_t)K * e.ld;
    const int64_t bytes = slots * 12 + e.ld * 4;
    const int64_t cap = resolve_cap(h->params);
    if (bytes > cap)
        return set_error(SPMV_ERR_TOO_LARGE, "ELL part of %lld x %d slots needs %lld bytes, cap %lld", (long long)e.ld,
                         K, (long long)bytes, (long long)cap);
    const std::string pre = hyb ? "ell_" : "";
    SPMV_TRY(h->alloc(&e.row_len, (size_t)e.ld, (pre + "row_len").c_str()));
    SPMV_TRY(h->alloc(&e.col, (size_t)slots, (pre + "col").c_str()));
    SPMV_TRY(h->alloc(&e.val, (size_t)slots, (pre + "val").c_str()));
    SPMV_CUDA(cudaMemsetAsync(e.row_len, 0, sizeof(int32_t) * (size_t)e.ld, s));
    if (slots > 0) {
        SPMV_CUDA(cudaMemsetAsync(e.col, 0, sizeof(int32_t) * (size_t)slots, s));
        SPMV_CUDA(cudaMemsetAsync(e.val, 0, sizeof(double) * (size_t)slots, s));
    }
    k_ell_row_len<<<grid_for(m, 256), 256, 0, s>>>(len, m, K, e.row_len);
    if (c->nnz > 0 && K > 0) {
        int g = grid_capped(c->nnz, 256, 64);
        k_ell_scatter<<<g, 256, 0, s>>>(c->ptr, c->idx, c->val, m, c->nnz, K, e.ld, e.col, e.val);
    }
    SPMV_CUDA(cudaGetLastError());
    h->stored_slots += slots;
    e.n_long = 0;
    return SPMV_OK;
}

// Threshold above which an ELL row is processed by a whole block.
static int32_t ell_long_threshold(const spmv_handle* h) {
    const int64_t avg = h->m > 0 ? ceil_div(h->nnz, h->m) : 0;
    const int64_t t = 4 * avg > kEllLongRow ? 4 * avg : kEllLongRow;
    return (int32_t)t;
}

int ell_convert(spmv_handle* h, const spmv_csr* c, cudaStream_t s) {
    Scratch tmp;
    int32_t* len = nullptr;
    SPMV_TRY(tmp.get(&len, (size_t)c->m + 1));
    SPMV_TRY(row_lengths(c->ptr, c->m, len, s));
    int32_t K = 0;
    SPMV_TRY(max_i32(len, c->m, &K, s, tmp));
    SPMV_TRY(ell_build(h, h->ell, c, K, len, false, s));
    // long rows: compaction of rows with row_len > threshold
    const int32_t thr = ell_long_threshold(h);
    int32_t *f = nullptr, *off = nullptr;
    SPMV_TRY(tmp.get(&f, (size_t)c->m + 1));
    SPMV_TRY(tmp.get(&off, (size_t)c->m + 2));
    k_flag_long<<<grid_for((int64_t)c->m + 1, 256), 256, 0, s>>>(h->ell.row_len, c->m, thr, f);
    SPMV_CUDA(cudaGetLastError());
    SPMV_TRY(exclusive_scan<int32_t>(f, off, (int64_t)c->m + 1, s, tmp));
    int32_t nl = 0;
    SPMV_CUDA(cudaMemcpyAsync(&nl, off + c->m, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA(cudaStreamSynchronize(s));
    h->ell.n_long = nl;
    SPMV_TRY(h->alloc(&h->ell.long_rows, (size_t)(nl > 0 ? nl : 1), "long_rows"));
    if (nl > 0) k_compact<<<grid_for(c->m, 256), 256, 0, s>>>(f, off, c->m, h->ell.long_rows);
    SPMV_CUDA(cudaGetLastError());
    SPMV_CUDA(cudaStreamSynchronize(s));
    h->aux[0] = K;
    h->aux[1] = nl;
    h->aux[2] = thr;
    return SPMV_OK;
}

// Blocks [0, nb) take 512 rows each (2 per thread); blocks nb.. take one long row each.
__global__ void __launch_bounds__(256) k_ell(dev::EllArgs a, int32_t nb, const int32_t* __restrict__ long_rows) {
    __shared__ double red[8];
    dev::pdl_wait();  // launched early (launch_pdl): wait for the kernel ahead
    if ((int32_t)blockIdx.x < nb) {
        dev::ell_rows2(a, (int32_t)(blockIdx.x * 512 + threadIdx.x * 2));
    } else {
        dev::ell_long_row(a, long_rows[blockIdx.x - nb], red);
    }
}

int ell_launch(const EllPart& e, int32_t m, int32_t long_len, const double* x, double* y, cudaStream_t s) {
    dev::EllArgs a{e.row_len, e.col, e.val, e.ld, m, long_len, x, y};
    const int32_t nb = (int32_t)ceil_div(m, 512);
    launch_pdl(k_ell, dim3(nb + e.n_long), dim3(256), 0, s, a, nb, e.long_rows);
    SPMV_CUDA(cudaGetLastError());
    return SPMV_OK;
}

int ell_run(const spmv_handle* h, const double* x, double* y, cudaStream_t s) {
    return ell_launch(h->ell, h->m, (int32_t)h->aux[2], x, y, s);
}

__global__ void k_ell_gather(const int32_t* __restrict__ ptr, int32_t m, int64_t nnz, int64_t ld,
                             const int32_t* __restrict__ col, const double* __restrict__ ev, int32_t* __restrict__ idx,
                             double* __restrict__ val) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = row_of_nnz(ptr, m, k);
        const int64_t j = k - ptr[r];
        idx[k] = col[j * ld + r];
        val[k] = ev[j * ld + r];
    }
}

int ell_to_csr(const spmv_handle* h, int32_t* ptr, int32_t* idx, double* val, cudaStream_t s) {
    Scratch tmp;
    SPMV_TRY(exclusive_scan<int32_t>(h->ell.row_len, ptr, h->m, s, tmp));
    if (h->nnz > 0) {
        int g = grid_capped(h->nnz, 256, 64);
        k_ell_gather<<<g, 256, 0, s>>>(ptr, h->m, h->nnz, h->ell.ld, h->ell.col, h->ell.val, idx, val);
    }
    SPMV_CUDA(cudaGetLastError());
    SPMV_CUDA(cudaStreamSynchronize(s));
    return SPMV_OK;
}

}  // namespace spmv
