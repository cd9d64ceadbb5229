// CSR (Sec. II-B "CSR"): y_i = sum of val[k] * x[idx[k]] over row i's range.
// The handle keeps a copy of the CSR arrays plus warp work units (see
// build_csr_units); each warp of a 256-thread block processes one unit.
#include "internal.cuh"
#include "kernels.cuh"

namespace spmv {

template <bool ADD>
__global__ void __launch_bounds__(256) k_csr_units(dev::CsrArgs a, int32_t n_units) {
    __shared__ dev::CsrWarpSmem S[8];
    const int w = threadIdx.x >> 5;
    const int32_t u = (int32_t)(blockIdx.x * 8 + w);
    if (u < n_units) dev::csr_warp_unit<ADD>(a, u, S[w], threadIdx.x & 31);
}

int csr_units_launch(const CsrUnits& cu, const int32_t* ptr, const int32_t* idx, const double* val,
                     const int32_t* row_map, const double* x, double* y, bool add, cudaStream_t s) {
    if (cu.n <= 0) return SPMV_OK;
    dev::CsrArgs a{cu.units, ptr, idx, val, row_map, x, y, cu.partial, cu.counters};
    const int g = grid_for(cu.n, 8);
    if (add) k_csr_units<true><<<g, 256, 0, s>>>(a, cu.n);
    else k_csr_units<false><<<g, 256, 0, s>>>(a, cu.n);
    SPMV_CUDA(cudaGetLastError());
    return SPMV_OK;
}

int csr_convert(spmv_handle* h, const spmv_csr* c, cudaStream_t s) {
    if (h->params.csr_block_nnz != 0 && h->params.csr_block_nnz != dev::kCsrW)
        return set_error(SPMV_ERR_INVALID_ARG, "csr_block_nnz must be 0 or %d (got %d)", dev::kCsrW,
                         h->params.csr_block_nnz);
    h->params.csr_block_nnz = dev::kCsrW;
    SPMV_TRY(copy_csr(h, c, s));
    SPMV_TRY(build_csr_units(h, h->cu, h->ptr, h->m, "", s));
    h->stored_slots = h->nnz;
    h->aux[0] = h->cu.n;
    return SPMV_OK;
}

int csr_run(const spmv_handle* h, const double* x, double* y, cudaStream_t s) {
    return csr_units_launch(h->cu, h->ptr, h->idx, h->val, nullptr, x, y, false, s);
}

}  // namespace spmv
