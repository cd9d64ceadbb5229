// CSR (Sec. II-B "CSR"): y_i = sum of val[k] * x[idx[k]] over row i's range.
// The handle keeps a copy of the CSR arrays plus row-block work units (see
// build_csr_units); one 256-thread block processes one unit.
#include "internal.cuh"
#include "kernels.cuh"

namespace spmv {

template <bool ADD>
__global__ void __launch_bounds__(256) k_csr_units(dev::CsrArgs a, int32_t block_nnz) {
    extern __shared__ double smem[];
    __shared__ double red[8];
    dev::csr_unit<ADD>(a, (int32_t)blockIdx.x, smem, block_nnz, red);
}

int csr_units_launch(const CsrUnits& cu, const int32_t* ptr, const int32_t* idx, const double* val,
                     const int32_t* row_map, const double* x, double* y, bool add, cudaStream_t s) {
    if (cu.n <= 0) return SPMV_OK;
    dev::CsrArgs a{cu.units, ptr, idx, val, row_map, x, y, cu.partial, cu.counters, cu.chunk};
    const size_t smem = dev::csr_smem_bytes(cu.block_nnz);
    if (add) k_csr_units<true><<<cu.n, 256, smem, s>>>(a, cu.block_nnz);
    else k_csr_units<false><<<cu.n, 256, smem, s>>>(a, cu.block_nnz);
    SPMV_CUDA(cudaGetLastError());
    return SPMV_OK;
}

// Opt the CSR kernels into the shared memory of the largest block budget
// (called at conversion time, never while a stream is being captured).
int csr_prepare_kernels() {
    const int smem = (int)dev::csr_smem_bytes(2048);
    SPMV_CUDA(cudaFuncSetAttribute((const void*)k_csr_units<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    SPMV_CUDA(cudaFuncSetAttribute((const void*)k_csr_units<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    return SPMV_OK;
}

int csr_convert(spmv_handle* h, const spmv_csr* c, cudaStream_t s) {
    int32_t B = h->params.csr_block_nnz;
    if (B == 0) B = 512;
    if (B < 128 || B > 2048 || (B & (B - 1)))
        return set_error(SPMV_ERR_INVALID_ARG, "csr_block_nnz must be a power of two in [128, 2048] (got %d)", B);
    h->params.csr_block_nnz = B;
    SPMV_TRY(copy_csr(h, c, s));
    SPMV_TRY(build_csr_units(h, h->cu, h->ptr, h->m, B, "", s));
    h->stored_slots = h->nnz;
    h->aux[0] = h->cu.n;
    return SPMV_OK;
}

int csr_run(const spmv_handle* h, const double* x, double* y, cudaStream_t s) {
    return csr_units_launch(h->cu, h->ptr, h->idx, h->val, nullptr, x, y, false, s);
}

}  // namespace spmv
